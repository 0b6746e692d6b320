// blp_tune.cu -- launch settings of the wavefront kernel per handle, and an
// autotuner that picks them by timing the preconditioner (Sec. 3.1 / 3.2 as
// one application of M^-1) on the handle's own problem.
//
// The settings change how the downstream sweeps are scheduled, never what
// they compute (up to rounding order in the two-step form): rows per
// boundary hand-off, CTAs per thread-block cluster, and one- or two-step
// recurrence per precision.  Which is fastest depends on the block sizes
// (N), on the precision and on the device, so the batched solver tunes once
// per (N, precision) and caches the choice for the process.
#include "blp_common.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

namespace {

// deterministic right-hand side in the region layout (padding stays zero)
template <typename T>
__global__ void k_tune_fill(Layout lay, T *out) {
    const int M = lay.N - 1;
    const long long n = (long long)M * M;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % M) + 1, j = (int)(k / M) + 1;
        const unsigned x = (unsigned)k * 2654435761u;
        out[lay.addr(i, j)] = T((double)(x >> 8) * (2.0 / 16777216.0) - 1.0);
    }
}

bool valid(const blp_tuning &t) {
    return (t.dts_chunk == 0 || t.dts_chunk == 8 || t.dts_chunk == 16 || t.dts_chunk == 32) && t.dts_cluster >= 1 &&
           t.dts_cluster <= 16 && (t.two_step & ~3) == 0;
}

// graphs embed the launch shapes they were captured with: drop them, and run
// the next application of each kind eagerly again before capturing
void apply(blp_handle *h, const blp_tuning &t) {
    const bool same = h->dts_chunk == t.dts_chunk && h->dts_max_cluster == t.dts_cluster &&
                      h->dts_two_step32 == ((t.two_step & 1) != 0) && h->dts_two_step64 == ((t.two_step & 2) != 0);
    if (same) return;
    cudaStreamSynchronize(h->stream);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (auto &row : h->solve_graph)
        for (auto &g : row)
            if (g.exec) {
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
            }
    for (auto &w : h->warm) w[0] = w[1] = false;
    h->dts_chunk = t.dts_chunk;
    h->dts_max_cluster = t.dts_cluster;
    h->dts_two_step32 = (t.two_step & 1) != 0;
    h->dts_two_step64 = (t.two_step & 2) != 0;
}

blp_tuning current(const blp_handle *h) {
    blp_tuning t;
    t.dts_chunk = h->dts_chunk;
    t.dts_cluster = h->dts_max_cluster;
    t.two_step = (h->dts_two_step32 ? 1 : 0) | (h->dts_two_step64 ? 2 : 0);
    t.precond_ms = h->tuned_ms;
    return t;
}

// mean device time of `reps` preconditioner applications after two warm-up
// applications (the first runs eagerly, the second captures the graph)
template <typename T>
int time_precond(blp_handle *h, const T *v, T *z, int reps, double *ms) {
    int cyc = 0, rc;
    for (int w = 0; w < 2; w++)
        if ((rc = precond_apply<T>(h, v, z, 0, &cyc))) return rc;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaGetLastError();
        return BLP_ERR_CUDA;
    }
    rc = BLP_OK;
    if (cudaEventRecord(e0, h->stream) != cudaSuccess) rc = BLP_ERR_CUDA;
    for (int k = 0; k < reps && rc == BLP_OK; k++) rc = precond_apply<T>(h, v, z, 0, &cyc);
    float t = 0.f;
    if (rc == BLP_OK && (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = BLP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BLP_OK) {
        cudaGetLastError();
        return rc;
    }
    if ((rc = blp_internal_check_err(h))) return rc;
    *ms = (double)t / reps;
    return BLP_OK;
}

template <typename T>
int autotune(blp_handle *h, int reps, blp_tuning *best) {
    const long long np = h->lay.npad;
    T *v = nullptr, *z = nullptr;
    int rc = blp_internal_alloc(h, (void **)&v, sizeof(T) * np);
    if (rc == BLP_OK) rc = blp_internal_alloc(h, (void **)&z, sizeof(T) * np);
    if (rc == BLP_OK && cudaMemsetAsync(v, 0, sizeof(T) * np, h->stream) != cudaSuccess) rc = BLP_ERR_CUDA;
    if (rc == BLP_OK) {
        k_tune_fill<T><<<grid_for(np, 256), 256, 0, h->stream>>>(h->lay, v);
        if (cudaGetLastError() != cudaSuccess) rc = BLP_ERR_CUDA;
    }
    // candidates: cluster sizes only up to the widest block's strip count
    // (larger ones give the same launch); chunk lengths 8 / 16 / 32 (the
    // launch falls back to a shorter chunk where the stages do not fit);
    // the one- and two-step forms for this precision
    const int strips = (std::max(h->L, h->N - 1 - h->L) + 31) / 32;
    std::vector<int> clusters;
    for (int c : {2, 4, 8, 16})
        if (c == 2 || c / 2 < strips) clusters.push_back(c);
    const int bit = sizeof(T) == 4 ? 1 : 2;
    const blp_tuning start = current(h);
    blp_tuning top = start;
    top.precond_ms = -1.0;
    for (int chunk : {8, 16, 32}) {
        for (int cl : clusters) {
            for (int two : {0, 1}) {
                if (rc != BLP_OK) break;
                blp_tuning t = start;
                t.dts_chunk = chunk;
                t.dts_cluster = cl;
                t.two_step = two ? (start.two_step | bit) : (start.two_step & ~bit);
                apply(h, t);
                double ms = 0.0;
                rc = time_precond<T>(h, v, z, reps, &ms);
                if (rc == BLP_OK && (top.precond_ms < 0.0 || ms < top.precond_ms)) {
                    top = t;
                    top.precond_ms = ms;
                }
            }
        }
    }
    blp_internal_free(h, v);
    blp_internal_free(h, z);
    if (rc != BLP_OK) {
        apply(h, start);
        return rc;
    }
    apply(h, top);
    h->tuned_ms = top.precond_ms;
    if (best) *best = top;
    return BLP_OK;
}

std::mutex cache_mu;
std::map<std::pair<int, int>, blp_tuning> cache;   // (N, precision) -> chosen setting

}  // namespace

extern "C" int blp_get_tuning(blp_handle *h, blp_tuning *t) {
    if (!h || !t) return BLP_ERR_ARG;
    *t = current(h);
    return BLP_OK;
}

extern "C" int blp_set_tuning(blp_handle *h, const blp_tuning *t) {
    if (!h || !t || !valid(*t)) return BLP_ERR_ARG;
    apply(h, *t);
    return BLP_OK;
}

extern "C" int blp_autotune(blp_handle *h, int precision, int reps, blp_tuning *best) {
    if (!h || (precision != BLP_FP64 && precision != BLP_MIXED)) return BLP_ERR_ARG;
    if (reps <= 0) reps = 3;
    return precision == BLP_MIXED ? autotune<float>(h, reps, best) : autotune<double>(h, reps, best);
}

// Setting chosen for (N, precision) in this process, tuning it first on the
// given problem when there is none yet (used by blp_solve_batched_tuned);
// with null fields a lookup only (BLP_ERR_ARG when nothing is cached).
int blp_internal_cached_tuning(const blp_params *p, const double *c1, const double *c2, const double *r,
                               cudaStream_t s, blp_tuning *t) {
    const std::pair<int, int> key(p->N, p->precision == BLP_MIXED ? 1 : 0);
    {
        std::lock_guard<std::mutex> g(cache_mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *t = it->second;
            return BLP_OK;
        }
    }
    if (!c1 || !c2 || !r) return BLP_ERR_ARG;
    blp_handle *h = nullptr;
    int rc = blp_internal_setup(p, c1, c2, r, s, &h);
    if (rc == BLP_OK) {
        rc = blp_autotune(h, p->precision, 0, t);
        blp_destroy(h);
    }
    if (rc != BLP_OK) return rc;
    std::lock_guard<std::mutex> g(cache_mu);
    cache.emplace(key, *t);   // a concurrent tuning of the same key keeps the first result
    *t = cache.at(key);
    return BLP_OK;
}
