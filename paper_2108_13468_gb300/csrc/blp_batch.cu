// blp_batch.cu -- many independent problems (different N, eps, fields,
// right-hand sides) solved concurrently on one GPU.
//
// Each problem is the single-instance solve of Sec. 3.3 (FGMRES with the
// Sec. 3.1 preconditioner).  A problem keeps only a few SMs busy at a time
// (the wavefront cluster, the two line chains, small grid-stride kernels),
// so several problems run side by side: K host worker threads, each with
// its own non-blocking stream, take the next unsolved problem, set it up,
// solve it and release it.  Handles allocate from the library's
// stream-ordered pool, so no worker synchronises the device.  The tuned
// variant first autotunes the wavefront launch settings once per new
// (N, precision) pair (blp_tune.cu) and gives each problem its pair's.
#include "blp_common.cuh"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

namespace {

void run_worker(blp_batch_item *items, int count, std::atomic<int> *next, int device, bool tuned) {
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        for (int i; (i = next->fetch_add(1)) < count;) items[i].info.status = items[i].status = BLP_ERR_CUDA;
        return;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        for (int i; (i = next->fetch_add(1)) < count;) items[i].info.status = items[i].status = BLP_ERR_CUDA;
        return;
    }
    for (int i; (i = next->fetch_add(1)) < count;) {
        blp_batch_item &it = items[i];
        memset(&it.info, 0, sizeof(it.info));
        blp_handle *h = nullptr;
        int rc = blp_internal_setup(&it.params, it.c1, it.c2, it.r, s, &h);
        blp_tuning t;
        if (rc == BLP_OK && tuned && blp_internal_cached_tuning(&it.params, nullptr, nullptr, nullptr, s, &t) == BLP_OK)
            blp_set_tuning(h, &t);
        if (rc == BLP_OK) {
            rc = blp_solve(h, it.f, it.u, it.tol, &it.info);
            blp_destroy(h);
        }
        it.info.status = rc;
        it.status = rc;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
}

}  // namespace

static int solve_batched(blp_batch_item *items, int count, int concurrency, bool tuned) {
    if (count < 0 || (count > 0 && !items)) return BLP_ERR_ARG;
    if (count == 0) return BLP_OK;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return BLP_ERR_CUDA;
    }
    if (tuned) {
        // tune each new (N, precision) pair before any problem runs, one at a
        // time, so that no other work shares the device while it is timed
        cudaStream_t ts = nullptr;
        if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return BLP_ERR_CUDA;
        }
        blp_tuning t;
        for (int i = 0; i < count; i++)
            blp_internal_cached_tuning(&items[i].params, items[i].c1, items[i].c2, items[i].r, ts, &t);
        cudaStreamSynchronize(ts);
        cudaStreamDestroy(ts);
    }
    for (int i = 0; i < count; i++) items[i].status = -1;
    const int K = std::max(1, std::min(concurrency > 0 ? concurrency : 16, count));
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    try {
        for (int k = 1; k < K; k++) pool.emplace_back(run_worker, items, count, &next, device, tuned);
    } catch (...) {
        // fewer workers than asked: the ones running (and this thread) finish the batch
    }
    run_worker(items, count, &next, device, tuned);
    for (auto &t : pool) t.join();
    for (int i = 0; i < count; i++)
        if (items[i].status != BLP_OK) return items[i].status;
    return BLP_OK;
}

extern "C" int blp_solve_batched(blp_batch_item *items, int count, int concurrency) {
    return solve_batched(items, count, concurrency, false);
}

extern "C" int blp_solve_batched_tuned(blp_batch_item *items, int count, int concurrency) {
    return solve_batched(items, count, concurrency, true);
}
