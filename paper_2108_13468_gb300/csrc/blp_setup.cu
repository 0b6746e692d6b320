// blp_setup.cu -- mesh, assembly of the row-normalised operator, line
// factorisations, corner multigrid hierarchy, layout conversion and the
// handle life cycle.
#include "blp_common.cuh"
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <chrono>
#include <mutex>

// ---------------------------------------------------------------------------
// S0. Shishkin mesh (Sec. 2.2 eq. (tau 1D); Sec. 3 eq. (tau exponential)).
// ---------------------------------------------------------------------------
extern "C" double blp_mesh(int N, double eps, double sigma, double beta, double *x) {
    if (N < 8 || (N & 1) || !(eps > 0.0) || eps > 1.0 || !(beta > 0.0) || !(sigma > 0.0) || !x) return -1.0;
    double tau = sigma * eps * std::log((double)N) / beta;
    if (tau > 0.5) tau = 0.5;
    int m = N / 2;
    for (int i = 0; i <= m; i++) x[i] = ((double)i / (double)m) * tau;
    for (int i = m + 1; i <= N; i++) x[i] = tau + ((double)(i - m) / (double)m) * (1.0 - tau);
    x[0] = 0.0;
    x[N] = 1.0;
    return tau;
}

// Graded (Bakhvalov-Shishkin) layer mesh: the Shishkin tau, split and
// interior nodes; on [0, tau] the nodes sample the layer function
// exp(-beta x / (sigma eps)) at equal decrements 2 (1 - 1/N) / N.
extern "C" double blp_mesh_graded(int N, double eps, double sigma, double beta, double *x) {
    const double tau = blp_mesh(N, eps, sigma, beta, x);
    if (tau < 0.0 || tau >= 0.5) return tau;   // invalid, or the uniform mesh
    const int m = N / 2;
    const double scale = sigma * eps / beta, step = 2.0 * (1.0 - 1.0 / (double)N);
    for (int i = 1; i < m; i++) x[i] = -scale * std::log(1.0 - step * (double)i / (double)N);
    return tau;
}

// General Shishkin mesh (the Remark on general Shishkin meshes): NL of the N
// intervals on [0, tau], tau = min(NL/N, sigma eps ln N / beta).
extern "C" double blp_mesh_q(int N, int NL, double eps, double sigma, double beta, double *x) {
    if (N < 8 || NL < 1 || NL > N - 2 || !(eps > 0.0) || eps > 1.0 || !(beta > 0.0) || !(sigma > 0.0) || !x)
        return -1.0;
    const double q = (double)NL / (double)N;
    double tau = sigma * eps * std::log((double)N) / beta;
    if (tau > q) tau = q;
    for (int i = 0; i <= NL; i++) x[i] = ((double)i / (double)NL) * tau;
    for (int i = NL + 1; i <= N; i++) x[i] = tau + ((double)(i - NL) / (double)(N - NL)) * (1.0 - tau);
    x[0] = 0.0;
    x[NL] = tau;
    x[N] = 1.0;
    return tau;
}

// Parabolic-layer mesh in y (Sec. 3, eq. (tau parabolic)): tau = min(1/2,
// sigma sqrt(eps) ln N), N/2 equal intervals on each side of tau.
extern "C" double blp_mesh_parabolic(int N, double eps, double sigma, double *x) {
    if (N < 8 || (N & 1) || !(eps > 0.0) || eps > 1.0 || !(sigma > 0.0) || !x) return -1.0;
    double tau = sigma * std::sqrt(eps) * std::log((double)N);
    if (tau > 0.5) tau = 0.5;
    const int m = N / 2;
    for (int i = 0; i <= m; i++) x[i] = ((double)i / (double)m) * tau;
    for (int i = m + 1; i <= N; i++) x[i] = tau + ((double)(i - m) / (double)m) * (1.0 - tau);
    x[0] = 0.0;
    x[N] = 1.0;
    return tau;
}

extern "C" void blp_params_default(blp_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->eps = 1e-4; p->N = 128; p->sigma = 2.0; p->beta_x = 1.0; p->beta_y = 1.0;
    p->restart = 30; p->maxit = 20000; p->precision = BLP_FP64; p->stop_mode = BLP_STOP_SCALED;
    p->corner_reduction = 1e3; p->corner_max_cycles = 50; p->corner_fixed_cycles = 0;
    p->check_coefficients = 1;
    p->mesh = BLP_MESH_SHISHKIN;
}

extern "C" const char *blp_strerror(int s) {
    switch (s) {
    case BLP_OK: return "ok";
    case BLP_ERR_ARG: return "invalid argument";
    case BLP_ERR_COEF: return "coefficients violate c1 >= beta_x, c2 >= beta_y, r >= 0 or are not finite";
    case BLP_ERR_NOCONV: return "iteration limit reached before the tolerance";
    case BLP_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case BLP_ERR_CUDA: return "CUDA runtime error";
    case BLP_ERR_MEM: return "allocation failed";
    default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// S1. Upwind 5-point stencil (Sec. 3) on a tensor block, written into a
// region-major layout as the row-normalised couplings w = a / aC.
// Nodes (I,J), 1 <= I <= mx, 1 <= J <= my, coordinates xs[0..mx+1],
// ys[0..my+1]; fields read at standard-layout index ((J*st)-1)*(N-1) + (I*st)-1
// (st = 1 for the fine grid, 2^l for injection to corner level l).
// ---------------------------------------------------------------------------
struct AsmOut {
    int use_layout;       // 1: global Layout addressing, 0: single Region
    Layout lay;
    Region reg;
    double *aC;           // may be null
    double *wW, *wE, *wS, *wN;
    double *omega, *dfe;  // may be null
};

__global__ void k_assemble(int mx, int my, const double *__restrict__ xs, const double *__restrict__ ys,
                           double eps, const double *__restrict__ c1, const double *__restrict__ c2,
                           const double *__restrict__ r, int N, int st, AsmOut o) {
    long long n = (long long)mx * my;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int I = (int)(k % mx) + 1, J = (int)(k / mx) + 1;
        long long kf = (long long)(J * st - 1) * (N - 1) + (I * st - 1);
        double hi = xs[I] - xs[I - 1], hi1 = xs[I + 1] - xs[I];
        double hb = 0.5 * (hi + hi1);
        double kj = ys[J] - ys[J - 1], kj1 = ys[J + 1] - ys[J];
        double kb = 0.5 * (kj + kj1);
        double C1 = c1[kf], C2 = c2[kf], R = r[kf];
        double aW = -eps / (hb * hi);
        double aE = -eps / (hb * hi1) - C1 / hi1;
        double aS = -eps / (kb * kj);
        double aN = -eps / (kb * kj1) - C2 / kj1;
        double aC = eps / hb * (1.0 / hi + 1.0 / hi1) + eps / kb * (1.0 / kj + 1.0 / kj1) + C1 / hi1 + C2 / kj1 + R;
        long long p = o.use_layout ? o.lay.addr(I, J) : o.reg.addr(I - 1, J - 1);
        if (o.aC) o.aC[p] = aC;
        o.wW[p] = I > 1 ? aW / aC : 0.0;
        o.wE[p] = I < mx ? aE / aC : 0.0;
        o.wS[p] = J > 1 ? aS / aC : 0.0;
        o.wN[p] = J < my ? aN / aC : 0.0;
        if (o.omega) o.omega[p] = hb * kb * aC;
        if (o.dfe) o.dfe[p] = hb * kb;
    }
}

// Transposed-direction couplings: wET(i,j) = wE(i-1,j), wNT(i,j) = wN(i,j-1),
// wWT(i,j) = wW(i+1,j), wST(i,j) = wS(i,j+1).
struct TransArgs {
    int use_layout;
    Layout lay;
    Region reg;
    int mx, my;   // node block size (global: N-1 x N-1)
    const double *wW, *wE, *wS, *wN;
    double *wET, *wNT, *wWT, *wST;
};
__device__ __forceinline__ long long tr_addr(const TransArgs &t, int I, int J) {
    return t.use_layout ? t.lay.addr(I, J) : t.reg.addr(I - 1, J - 1);
}
__global__ void k_transpose_couplings(TransArgs t) {
    long long n = (long long)t.mx * t.my;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int I = (int)(k % t.mx) + 1, J = (int)(k / t.mx) + 1;
        long long p = tr_addr(t, I, J);
        t.wET[p] = I > 1 ? t.wE[tr_addr(t, I - 1, J)] : 0.0;
        t.wNT[p] = J > 1 ? t.wN[tr_addr(t, I, J - 1)] : 0.0;
        t.wWT[p] = I < t.mx ? t.wW[tr_addr(t, I + 1, J)] : 0.0;
        t.wST[p] = J < t.my ? t.wS[tr_addr(t, I, J + 1)] : 0.0;
    }
}

// Thomas factorisation of every line of the Y and X blocks (Sec. 3.1:
// M_YY lines of constant x, tridiagonal (S, C, N) in y; M_XX lines of
// constant y, tridiagonal (W, C, E) in x), for the line matrices T and T^T.
// One thread per line.  With unit diagonal, sub s_k, super t_k:
//   u_0 = 1, l_k = s_k / u_{k-1}, u_k = 1 - l_k t_{k-1}
//   lf_k = -l_k, lg_k = 1/u_k, lh_k = -t_k/u_k  (lh_{n-1} = 0)
__global__ void k_line_factors(Layout lay, const double *wW, const double *wE, const double *wS, const double *wN,
                               double *lf, double *lg, double *lh, double *lfT, double *lgT, double *lhT) {
    int L = lay.L;
    const Region &Y = lay.R[2], &X = lay.R[1];
    int nY = Y.mx, nX = X.my;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nY + nX) return;
    bool isY = t < nY;
    int line = isY ? t : t - nY;
    auto slot = [&](int k) -> long long { return isY ? Y.addr(line, k) : X.addr(k, line); };
    auto sub = [&](int k) -> double { return k > 0 ? (isY ? wS[slot(k)] : wW[slot(k)]) : 0.0; };
    auto sup = [&](int k) -> double { return k < L - 1 ? (isY ? wN[slot(k)] : wE[slot(k)]) : 0.0; };
    for (int pass = 0; pass < 2; pass++) {
        double *F = pass ? lfT : lf, *G = pass ? lgT : lg, *Hh = pass ? lhT : lh;
        double u_prev = 1.0, t_prev = 0.0;
        for (int k = 0; k < L; k++) {
            // T: sub s_k, sup t_k.   T^T: sub s'_k = t_{k-1}, sup t'_k = s_{k+1}
            double s = pass ? (k > 0 ? sup(k - 1) : 0.0) : sub(k);
            double tk = pass ? (k < L - 1 ? sub(k + 1) : 0.0) : sup(k);
            double l = k > 0 ? s / u_prev : 0.0;
            double u = k > 0 ? 1.0 - l * t_prev : 1.0;
            long long p = slot(k);
            F[p] = -l;
            G[p] = 1.0 / u;
            Hh[p] = -tk / u;
            u_prev = u;
            t_prev = tk;
        }
    }
}

// (a, b) -> packed pairs, in either precision
template <typename T>
__global__ void k_pack_pairs(const double *__restrict__ a, const double *__restrict__ b,
                             typename Pair2<T>::type *__restrict__ out, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        typename Pair2<T>::type v;
        v.x = (T)a[k];
        v.y = (T)b[k];
        out[k] = v;
    }
}

// skew-layout level arrays -> natural row-major copies (10 arrays of m*m)
struct NatSrc { const double *a[10]; };
__global__ void k_to_natural(Region R, NatSrc src, double *nat) {
    const int m = R.mx;
    const int n = m * m;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long p = R.addr(k % m, k / m);
        for (int q = 0; q < 10; q++) nat[(long long)q * n + k] = src.a[q][p];
    }
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

// Standard (x-fastest) <-> region-major.  scale_mode: 0 none, 1 divide by
// aC, 2 multiply by aC (aC in region layout).
__global__ void k_std_to_region(Layout lay, const double *__restrict__ in, double *__restrict__ out,
                                const double *__restrict__ aC, int scale_mode) {
    int M = lay.N - 1;
    long long n = (long long)M * M;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int i = (int)(k % M) + 1, j = (int)(k / M) + 1;
        long long p = lay.addr(i, j);
        double v = in[k];
        if (scale_mode == 1) v /= aC[p];
        else if (scale_mode == 2) v *= aC[p];
        out[p] = v;
    }
}
__global__ void k_region_to_std(Layout lay, const double *__restrict__ in, double *__restrict__ out,
                                const double *__restrict__ aC, int scale_mode) {
    int M = lay.N - 1;
    long long n = (long long)M * M;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        int i = (int)(k % M) + 1, j = (int)(k / M) + 1;
        long long p = lay.addr(i, j);
        double v = in[p];
        if (scale_mode == 1) v /= aC[p];
        else if (scale_mode == 2) v *= aC[p];
        out[k] = v;
    }
}

// coefficient validation: red[0] = min(c1 - bx), red[1] = min(c2 - by),
// red[2] = min r, flags: nonfinite
__global__ void k_check_coefs(const double *c1, const double *c2, const double *r, long long n, double bx,
                              double by, double *out /* 3 per block */, int *nonfinite) {
    double m0 = 1e300, m1 = 1e300, m2 = 1e300;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double a = c1[k], b = c2[k], c = r[k];
        if (!isfinite(a) || !isfinite(b) || !isfinite(c)) atomicExch(nonfinite, 1);
        m0 = fmin(m0, a - bx); m1 = fmin(m1, b - by); m2 = fmin(m2, c);
    }
    __shared__ double s[3][256];
    s[0][threadIdx.x] = m0; s[1][threadIdx.x] = m1; s[2][threadIdx.x] = m2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; q++) s[q][threadIdx.x] = fmin(s[q][threadIdx.x], s[q][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) out[blockIdx.x * 3 + q] = s[q][0];
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Device memory of a handle comes from one library-owned stream-ordered
// pool per device: allocations and frees are ordered on the handle's
// stream and never synchronise the device, so handles on different streams
// (the batched solver) run concurrently; up to 4 GiB of freed memory stays
// in the pool for reuse.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static int lib_pool(cudaMemPool_t *out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return BLP_ERR_CUDA; }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { cudaGetLastError(); return BLP_ERR_CUDA; }
        unsigned long long keep = 4ULL << 30;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolDestroy(pool);
            return BLP_ERR_CUDA;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return BLP_OK;
}

int blp_internal_alloc(blp_handle *h, void **p, size_t bytes) {
    cudaMemPool_t pool;
    *p = nullptr;
    int rc = lib_pool(&pool);
    if (rc != BLP_OK) return rc;
    if (cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, h->stream) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return BLP_ERR_MEM;
    }
    return BLP_OK;
}

void blp_internal_free(blp_handle *h, void *p) {
    if (p && cudaFreeAsync(p, h->stream) != cudaSuccess) cudaGetLastError();
}

// Page-locked host mirrors of DevState, recycled across handles (page-locked
// allocation would synchronise the device).
static std::mutex g_pinned_mu;
static std::vector<DevState *> g_pinned_free;

static DevState *pinned_get() {
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            DevState *d = g_pinned_free.back();
            g_pinned_free.pop_back();
            return d;
        }
    }
    DevState *d = nullptr;
    if (cudaMallocHost((void **)&d, sizeof(DevState)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return d;
}
static void pinned_put(DevState *d) {
    if (!d) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back(d);
}

template <typename T>
static int dalloc(blp_handle *h, T **p, long long n) {
    void *q = nullptr;
    int rc = blp_internal_alloc(h, &q, sizeof(T) * (size_t)(n > 0 ? n : 1));
    *p = static_cast<T *>(q);
    return rc;
}

#define TRY(x) do { int rc_ = (x); if (rc_ != BLP_OK) return rc_; } while (0)

template <typename T>
static void free_coefs(blp_handle *h, Coefs<T> &c) {
    blp_internal_free(h, c.pF);
    blp_internal_free(h, c.pR);
    T *ps[] = {c.wW, c.wE, c.wS, c.wN, c.wET, c.wNT, c.wWT, c.wST, c.lf, c.lg, c.lh, c.lfT, c.lgT, c.lhT,
               c.cpre, c.cpreT};
    for (T *p : ps) blp_internal_free(h, p);
    c = Coefs<T>();
}
template <typename T>
static void free_hier(blp_handle *h, Hierarchy<T> &H) {
    for (int l = 0; l < H.nlev; l++) {
        Level<T> &v = H.lev[l];
        blp_internal_free(h, v.pF);
        blp_internal_free(h, v.pR);
        blp_internal_free(h, v.beta);
        blp_internal_free(h, v.nat);
        T *ps[] = {v.wW, v.wE, v.wS, v.wN, v.wET, v.wNT, v.wWT, v.wST, v.omega, v.dfe, v.e[0], v.e[1], v.b};
        for (T *p : ps) blp_internal_free(h, p);
        v = Level<T>();
    }
    H.nlev = 0;
}

extern "C" void blp_destroy(blp_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_coefs(h, h->cd);
    free_coefs(h, h->cf);
    free_hier(h, h->hd);
    free_hier(h, h->hf);
    blp_internal_semi_free(h);
    blp_internal_prof_flush(h);
    for (auto &e : h->prof.ev) cudaEventDestroy(e);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (auto &row : h->solve_graph)
        for (auto &g : row)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaStream_t &cs : h->cap)
        if (cs) cudaStreamDestroy(cs);
    for (int q = 0; q < 2; q++) { blp_internal_free(h, h->gv[q]); blp_internal_free(h, h->gz[q]); }
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    void *ps[] = {h->x, h->y, h->aC, h->c1, h->c2, h->r, h->partials, h->dev, h->err, h->ws,
                  h->stage[0], h->stage[1], h->stage[2], h->stage[3]};
    for (void *p : ps) blp_internal_free(h, p);
    pinned_put(h->host_state);
    cudaStreamSynchronize(h->stream);
    delete h;
}

extern "C" int blp_set_stream(blp_handle *h, void *stream) {
    if (!h) return BLP_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return BLP_OK;
}

extern "C" long long blp_kernel_launches(const blp_handle *h) { return h ? h->launches : -1; }

int blp_internal_prof_flush(blp_handle *h) {
    ProfState &P = h->prof;
    if (P.used == 0) return BLP_OK;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < P.used; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]) == cudaSuccess) {
            P.count[P.cls[i]]++;
            P.ms[P.cls[i]] += ms;
        } else {
            cudaGetLastError();
        }
    }
    P.used = 0;
    return BLP_OK;
}

extern "C" int blp_profile(blp_handle *h, int enable) {
    if (!h) return BLP_ERR_ARG;
    ProfState &P = h->prof;
    if (enable) {
        if (P.ev.empty()) {
            P.ev.resize(2 * 4096);
            P.cls.resize(4096);
            for (auto &e : P.ev) CUDA_TRY(cudaEventCreate(&e));
        }
        for (int c = 0; c < KC_COUNT; c++) { P.count[c] = 0; P.ms[c] = 0.0; P.bytes[c] = 0.0; P.steps[c] = 0.0; }
        P.used = 0;
        P.on = true;
    } else {
        int rc = blp_internal_prof_flush(h);
        P.on = false;
        return rc;
    }
    return BLP_OK;
}

extern "C" int blp_profile_chain_steps(blp_handle *h, int cls, double *steps) {
    if (!h || cls < 0 || cls >= KC_COUNT || !steps) return BLP_ERR_ARG;
    *steps = h->prof.steps[cls];
    return BLP_OK;
}

extern "C" int blp_profile_read(blp_handle *h, int cls, long long *count, double *total_ms, double *bytes) {
    if (!h || cls < 0 || cls >= KC_COUNT) return BLP_ERR_ARG;
    int rc = blp_internal_prof_flush(h);
    if (rc) return rc;
    if (count) *count = h->prof.count[cls];
    if (total_ms) *total_ms = h->prof.ms[cls];
    if (bytes) *bytes = h->prof.bytes[cls];
    return BLP_OK;
}

extern "C" int blp_kernel_class_count(void) { return KC_COUNT; }

extern "C" const char *blp_kernel_class_name(int cls) {
    static const char *names[KC_COUNT] = {"dts_gs", "dts_interior", "line_chain", "mg_restrict", "mg_prolong",
                                          "corner_norm", "matvec", "multidot", "update", "small", "layout", "gs_rhs",
                                          "mg_coarse"};
    return (cls >= 0 && cls < KC_COUNT) ? names[cls] : "";
}

int blp_internal_ensure_ws(blp_handle *h, size_t bytes) {
    if (h->ws_bytes >= bytes) return BLP_OK;
    if (h->ws) { blp_internal_free(h, h->ws); h->ws = nullptr; h->ws_bytes = 0; }
    int rc = blp_internal_alloc(h, &h->ws, bytes);
    if (rc != BLP_OK) return rc;
    h->ws_bytes = bytes;
    return BLP_OK;
}

int blp_internal_to_region(blp_handle *h, const double *in, double *out, int scale_mode) {
    CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * h->lay.npad, h->stream));
    long long n = (long long)(h->N - 1) * (h->N - 1);
    k_std_to_region<<<grid_for(n, 256), 256, 0, h->stream>>>(h->lay, in, out, h->aC, scale_mode);
    LAUNCH_CHECK(h);
    return BLP_OK;
}
int blp_internal_from_region(blp_handle *h, const double *in, double *out, int scale_mode) {
    long long n = (long long)(h->N - 1) * (h->N - 1);
    k_region_to_std<<<grid_for(n, 256), 256, 0, h->stream>>>(h->lay, in, out, h->aC, scale_mode);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

template <typename T>
static int alloc_coefs(blp_handle *h, Coefs<T> &c, long long n) {
    T **ps[] = {&c.wW, &c.wE, &c.wS, &c.wN, &c.wET, &c.wNT, &c.wWT, &c.wST, &c.lf, &c.lg, &c.lh, &c.lfT, &c.lgT, &c.lhT};
    for (T **p : ps) {
        TRY(dalloc(h, p, n));
        if (cudaMemsetAsync(*p, 0, sizeof(T) * n, h->stream) != cudaSuccess) return BLP_ERR_CUDA;
    }
    return BLP_OK;
}

template <typename T>
static int make_pairs(blp_handle *h, const double *wE, const double *wN, const double *wET, const double *wNT,
                      typename Pair2<T>::type **pF, typename Pair2<T>::type **pR, long long n) {
    TRY(dalloc(h, pF, n));
    TRY(dalloc(h, pR, n));
    k_pack_pairs<T><<<grid_for(n, 256), 256, 0, h->stream>>>(wE, wN, *pF, n);
    LAUNCH_CHECK(h);
    k_pack_pairs<T><<<grid_for(n, 256), 256, 0, h->stream>>>(wET, wNT, *pR, n);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

static int convert_coefs(blp_handle *h, long long n) {
    TRY(make_pairs<double>(h, h->cd.wE, h->cd.wN, h->cd.wET, h->cd.wNT, &h->cd.pF, &h->cd.pR, n));
    TRY(make_pairs<float>(h, h->cd.wE, h->cd.wN, h->cd.wET, h->cd.wNT, &h->cf.pF, &h->cf.pR, n));
    double *src[] = {h->cd.wW, h->cd.wE, h->cd.wS, h->cd.wN, h->cd.wET, h->cd.wNT, h->cd.wWT, h->cd.wST,
                     h->cd.lf, h->cd.lg, h->cd.lh, h->cd.lfT, h->cd.lgT, h->cd.lhT};
    float *dst[] = {h->cf.wW, h->cf.wE, h->cf.wS, h->cf.wN, h->cf.wET, h->cf.wNT, h->cf.wWT, h->cf.wST,
                    h->cf.lf, h->cf.lg, h->cf.lh, h->cf.lfT, h->cf.lgT, h->cf.lhT};
    for (int q = 0; q < 14; q++) {
        k_to_float<<<grid_for(n, 256), 256, 0, h->stream>>>(src[q], dst[q], n);
        LAUNCH_CHECK(h);
    }
    return BLP_OK;
}

// Corner hierarchy (Sec. 3.2): level l keeps the fine corner nodes whose
// index is a multiple of 2^l, the transition node on every level, the node
// outside the corner at the fine spacing H; fields injected; the operator
// re-discretised with the same stencil.  Coarsening stops when the side is
// odd or below 4.
static int build_hierarchy(blp_handle *h) {
    int L = h->L;
    std::vector<int> ms;
    int m = L;
    for (;;) {
        ms.push_back(m);
        if ((m & 1) || m < 4 || (int)ms.size() >= BLP_MAXLEV) break;
        m /= 2;
    }
    int nlev = (int)ms.size();
    h->hd.nlev = h->hf.nlev = nlev;
    double *dxs = nullptr, *dys = nullptr;
    TRY(dalloc(h, &dxs, L + 2));
    TRY(dalloc(h, &dys, L + 2));
    std::vector<double> xs(L + 2), ys(L + 2);
    for (int l = 0; l < nlev; l++) {
        int ml = ms[l], st = 1 << l;
        xs[0] = h->hx[0]; ys[0] = h->hy[0];
        for (int I = 1; I <= ml; I++) { xs[I] = h->hx[I * st]; ys[I] = h->hy[I * st]; }
        xs[ml + 1] = h->hx[L + 1]; ys[ml + 1] = h->hy[L + 1];
        CUDA_TRY(cudaMemcpyAsync(dxs, xs.data(), sizeof(double) * (ml + 2), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaMemcpyAsync(dys, ys.data(), sizeof(double) * (ml + 2), cudaMemcpyHostToDevice, h->stream));
        Level<double> &D = h->hd.lev[l];
        Level<float> &F = h->hf.lev[l];
        D.R = F.R = make_region(LAYOUT_SKEW, ml, ml, 1, 1, 0);
        long long n = D.R.size;
        double **pd[] = {&D.wW, &D.wE, &D.wS, &D.wN, &D.wET, &D.wNT, &D.wWT, &D.wST, &D.omega, &D.dfe, &D.e[0], &D.e[1], &D.b};
        float **pf[] = {&F.wW, &F.wE, &F.wS, &F.wN, &F.wET, &F.wNT, &F.wWT, &F.wST, &F.omega, &F.dfe, &F.e[0], &F.e[1], &F.b};
        for (int q = 0; q < 13; q++) {
            TRY(dalloc(h, pd[q], n));
            TRY(dalloc(h, pf[q], n));
            CUDA_TRY(cudaMemsetAsync(*pd[q], 0, sizeof(double) * n, h->stream));
            CUDA_TRY(cudaMemsetAsync(*pf[q], 0, sizeof(float) * n, h->stream));
        }
        AsmOut o;
        memset(&o, 0, sizeof(o));
        o.use_layout = 0; o.reg = D.R; o.aC = nullptr;
        o.wW = D.wW; o.wE = D.wE; o.wS = D.wS; o.wN = D.wN; o.omega = D.omega; o.dfe = D.dfe;
        k_assemble<<<grid_for((long long)ml * ml, 256), 256, 0, h->stream>>>(ml, ml, dxs, dys, h->p.eps, h->c1, h->c2,
                                                                          h->r, h->N, st, o);
        LAUNCH_CHECK(h);
        TransArgs t;
        memset(&t, 0, sizeof(t));
        t.use_layout = 0; t.reg = D.R; t.mx = ml; t.my = ml;
        t.wW = D.wW; t.wE = D.wE; t.wS = D.wS; t.wN = D.wN;
        t.wET = D.wET; t.wNT = D.wNT; t.wWT = D.wWT; t.wST = D.wST;
        k_transpose_couplings<<<grid_for((long long)ml * ml, 256), 256, 0, h->stream>>>(t);
        LAUNCH_CHECK(h);
        for (int q = 0; q < 10; q++) {
            k_to_float<<<grid_for(n, 256), 256, 0, h->stream>>>(*pd[q], *pf[q], n);
            LAUNCH_CHECK(h);
        }
        TRY(make_pairs<double>(h, D.wE, D.wN, D.wET, D.wNT, &D.pF, &D.pR, n));
        TRY(make_pairs<float>(h, D.wE, D.wN, D.wET, D.wNT, &F.pF, &F.pR, n));
        TRY(dalloc(h, &D.beta, n));
        TRY(dalloc(h, &F.beta, n));
        CUDA_TRY(cudaMemsetAsync(D.beta, 0, sizeof(double) * n, h->stream));
        CUDA_TRY(cudaMemsetAsync(F.beta, 0, sizeof(float) * n, h->stream));
        if (ml <= BLP_COARSE_MAX) {
            const long long nn = 10LL * ml * ml;
            TRY(dalloc(h, &D.nat, nn));
            TRY(dalloc(h, &F.nat, nn));
            NatSrc src = {{D.wW, D.wE, D.wS, D.wN, D.wET, D.wWT, D.wNT, D.wST, D.omega, D.dfe}};
            k_to_natural<<<grid_for((long long)ml * ml, 256), 256, 0, h->stream>>>(D.R, src, D.nat);
            LAUNCH_CHECK(h);
            k_to_float<<<grid_for(nn, 256), 256, 0, h->stream>>>(D.nat, F.nat, nn);
            LAUNCH_CHECK(h);
        }
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    blp_internal_free(h, dxs);
    blp_internal_free(h, dys);
    return BLP_OK;
}

static int setup_impl(blp_handle *h, const double *c1, const double *c2, const double *r) {
    const blp_params &p = h->p;
    int N = p.N;
    long long n = (long long)(N - 1) * (N - 1);
    h->N = N;
    h->L = p.layer_intervals > 0 ? p.layer_intervals : N / 2;
    h->lay = make_layout(N, h->L);
    long long np = h->lay.npad;
    h->hx.resize(N + 1);
    h->hy.resize(N + 1);
    auto mesh = p.mesh == BLP_MESH_GRADED ? blp_mesh_graded : blp_mesh;
    if (h->L != N / 2) {   // general Shishkin mesh, NL = h->L intervals in the layer
        h->tau_x = blp_mesh_q(N, h->L, p.eps, p.sigma, p.beta_x, h->hx.data());
        h->tau_y = blp_mesh_q(N, h->L, p.eps, p.sigma, p.beta_y, h->hy.data());
    } else {
        h->tau_x = mesh(N, p.eps, p.sigma, p.beta_x, h->hx.data());
        h->tau_y = p.mesh == BLP_MESH_PARABOLIC ? blp_mesh_parabolic(N, p.eps, p.sigma, h->hy.data())
                                                : mesh(N, p.eps, p.sigma, p.beta_y, h->hy.data());
    }
    TRY(dalloc(h, &h->x, N + 1));
    TRY(dalloc(h, &h->y, N + 1));
    CUDA_TRY(cudaMemcpyAsync(h->x, h->hx.data(), sizeof(double) * (N + 1), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->y, h->hy.data(), sizeof(double) * (N + 1), cudaMemcpyHostToDevice, h->stream));
    TRY(dalloc(h, &h->c1, n));
    TRY(dalloc(h, &h->c2, n));
    TRY(dalloc(h, &h->r, n));
    CUDA_TRY(cudaMemcpyAsync(h->c1, c1, sizeof(double) * n, cudaMemcpyDefault, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->c2, c2, sizeof(double) * n, cudaMemcpyDefault, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->r, r, sizeof(double) * n, cudaMemcpyDefault, h->stream));
    TRY(dalloc(h, &h->partials, BLP_SCALARS_OFF + 64));
    TRY(dalloc(h, &h->dev, 1));
    TRY(dalloc(h, &h->err, 4));
    CUDA_TRY(cudaMemsetAsync(h->dev, 0, sizeof(DevState), h->stream));
    CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int) * 4, h->stream));
    if (!(h->host_state = pinned_get())) return BLP_ERR_MEM;
    for (int q = 0; q < 4; q++) TRY(dalloc(h, &h->stage[q], n));

    if (p.check_coefficients) {
        int nb = 128;
        double *out = h->partials;
        int *nf = h->err + 1;
        // parabolic case: no convection in y is required (c2 >= 0)
        const double by = p.mesh == BLP_MESH_PARABOLIC ? 0.0 : p.beta_y;
        k_check_coefs<<<nb, 256, 0, h->stream>>>(h->c1, h->c2, h->r, n, p.beta_x, by, out, nf);
        LAUNCH_CHECK(h);
        std::vector<double> mins(3 * nb);
        int nonfinite = 0;
        CUDA_TRY(cudaMemcpyAsync(mins.data(), out, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(&nonfinite, nf, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        double m0 = 1e300, m1 = 1e300, m2 = 1e300;
        for (int b = 0; b < nb; b++) { m0 = fmin(m0, mins[3 * b]); m1 = fmin(m1, mins[3 * b + 1]); m2 = fmin(m2, mins[3 * b + 2]); }
        CUDA_TRY(cudaMemsetAsync(nf, 0, sizeof(int), h->stream));
        if (nonfinite || m0 < 0.0 || m1 < 0.0 || m2 < 0.0) return BLP_ERR_COEF;
    }

    TRY(dalloc(h, &h->aC, np));
    CUDA_TRY(cudaMemsetAsync(h->aC, 0, sizeof(double) * np, h->stream));
    TRY(alloc_coefs(h, h->cd, np));
    TRY(alloc_coefs(h, h->cf, np));
    AsmOut o;
    memset(&o, 0, sizeof(o));
    o.use_layout = 1; o.lay = h->lay; o.aC = h->aC;
    o.wW = h->cd.wW; o.wE = h->cd.wE; o.wS = h->cd.wS; o.wN = h->cd.wN;
    k_assemble<<<grid_for(n, 256), 256, 0, h->stream>>>(N - 1, N - 1, h->x, h->y, p.eps, h->c1, h->c2, h->r, N, 1, o);
    LAUNCH_CHECK(h);
    TransArgs t;
    memset(&t, 0, sizeof(t));
    t.use_layout = 1; t.lay = h->lay; t.mx = N - 1; t.my = N - 1;
    t.wW = h->cd.wW; t.wE = h->cd.wE; t.wS = h->cd.wS; t.wN = h->cd.wN;
    t.wET = h->cd.wET; t.wNT = h->cd.wNT; t.wWT = h->cd.wWT; t.wST = h->cd.wST;
    k_transpose_couplings<<<grid_for(n, 256), 256, 0, h->stream>>>(t);
    LAUNCH_CHECK(h);
    int nlines = h->lay.R[2].mx + h->lay.R[1].my;
    k_line_factors<<<(nlines + 127) / 128, 128, 0, h->stream>>>(h->lay, h->cd.wW, h->cd.wE, h->cd.wS, h->cd.wN,
                                                                h->cd.lf, h->cd.lg, h->cd.lh, h->cd.lfT, h->cd.lgT, h->cd.lhT);
    LAUNCH_CHECK(h);
    TRY(convert_coefs(h, np));
    TRY(blp_internal_chain_pre(h));
    TRY(build_hierarchy(h));
    if (p.mesh == BLP_MESH_PARABOLIC) TRY(blp_internal_semi_build(h));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return BLP_OK;
}

int blp_internal_setup(const blp_params *p, const double *c1, const double *c2, const double *r, cudaStream_t stream,
                       blp_handle **out) {
    if (!out) return BLP_ERR_ARG;
    *out = nullptr;
    if (!p || !c1 || !c2 || !r) return BLP_ERR_ARG;
    if (p->N < 8 || p->N > 16384 || (p->N & 1) || !(p->eps > 0.0) || p->eps > 1.0 || !(p->sigma > 0.0) ||
        !(p->beta_x > 0.0) || !(p->beta_y > 0.0) || p->restart < 1 || p->restart > 64 || p->maxit < 1 ||
        (p->precision != BLP_FP64 && p->precision != BLP_MIXED) || p->stop_mode < 0 || p->stop_mode > 2 ||
        !(p->corner_reduction >= 1.0) || p->corner_max_cycles < 1 ||
        (p->mesh != BLP_MESH_SHISHKIN && p->mesh != BLP_MESH_GRADED && p->mesh != BLP_MESH_PARABOLIC) ||
        p->layer_intervals < 0 || p->layer_intervals > p->N - 2 ||
        (p->layer_intervals > 0 && p->layer_intervals != p->N / 2 && p->mesh != BLP_MESH_SHISHKIN))
        return BLP_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    blp_handle *h = new blp_handle();
    h->p = *p;
    // tuning override: CTAs per wavefront cluster (1 = single-SM wavefront)
    if (const char *e = getenv("BLP_DTS_CLUSTER")) h->dts_max_cluster = std::max(1, std::min(16, atoi(e)));
    if (const char *e = getenv("BLP_DTS_TWO_STEP")) {   // bit 0: FP32 sweeps, bit 1: FP64 sweeps
        const int v = atoi(e);
        h->dts_two_step32 = (v & 1) != 0;
        h->dts_two_step64 = (v & 2) != 0;
    }
    if (const char *e = getenv("BLP_DTS_CHUNK")) {
        const int c = atoi(e);
        h->dts_chunk = (c == 8 || c == 16 || c == 32) ? c : 0;
    }
    if (const char *e = getenv("BLP_GRAPHS")) h->use_graphs = atoi(e) != 0;
    h->solve_graphs = p->device_driven != 0;
    if (const char *e = getenv("BLP_SOLVE_GRAPH")) h->solve_graphs = atoi(e) != 0;
    h->stream = stream;
    int rc = setup_impl(h, c1, c2, r);
    if (rc != BLP_OK) {
        blp_destroy(h);
        return rc;
    }
    h->t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return BLP_OK;
}

extern "C" int blp_setup(const blp_params *p, const double *c1, const double *c2, const double *r, blp_handle **out) {
    return blp_internal_setup(p, c1, c2, r, 0, out);
}

// Debug/inspection helpers for the host-side layout tests (no GPU needed).
extern "C" long long blp_layout_npad(int N) { return (N >= 8 && !(N & 1)) ? make_layout(N).npad : -1; }
extern "C" long long blp_layout_addr(int N, int i, int j) {
    if (N < 8 || (N & 1) || i < 1 || j < 1 || i > N - 1 || j > N - 1) return -1;
    return make_layout(N).addr(i, j);
}
extern "C" int blp_layout_node(int N, long long p, int *i, int *j) {
    if (N < 8 || (N & 1)) return -1;
    Layout L = make_layout(N);
    if (p < 0 || p >= L.npad) return -1;
    if (p >= L.R[3].off + L.R[3].size) return 0;
    return L.node(p, *i, *j) ? 1 : 0;
}
