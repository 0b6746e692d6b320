// blp_krylov.cu -- restarted flexible GMRES (Sec. 3.3) on the row-normalised
// system D^-1 A u = D^-1 f (D = diag(A)) with the FP64 or the FP32
// preconditioner, the adjoint solve and the gradient assembly; C-ABI entry
// points.
#include "blp_common.cuh"
#include <cstdint>
#include <type_traits>
#include <cmath>
#include <chrono>
#include <algorithm>

#define FULL 0xffffffffu
#define MAXV BLP_PART_STRIDE   // restart + 1 <= 65

// ---------------------------------------------------------------------------
// Operator of the normalised system (unit diagonal, Sec. 3 stencil / aC):
//   forward  y = x + wW x_W + wE x_E + wS x_S + wN x_N
//   adjoint  y = x + wET x_W + wWT x_E + wNT x_S + wST x_N   ((D^-1 A)^T)
// mode 0: out = Op x;  mode 1: out = f - Op x.  Padding slots get 0.
// ---------------------------------------------------------------------------
// xs != null (captured solve): also store x into column *jdev of xs.
template <typename TC, typename TX, typename TO, bool TRANS>
__global__ void k_matvec(Layout lay, Coefs<TC> c, const TX *__restrict__ x, TO *__restrict__ out,
                         const TO *__restrict__ f, int mode, const double *__restrict__ rs,
                         TX *__restrict__ xs = nullptr, const int *jdev = nullptr) {
    const int M = lay.N - 1;
    TX *const xcol = xs ? xs + (long long)*jdev * lay.npad : nullptr;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < lay.npad; p += (long long)gridDim.x * blockDim.x) {
        if (xcol) xcol[p] = x[p];
        int i, j;
        if (!lay.node(p, i, j)) { out[p] = TO(0); continue; }
        TO s = (TO)x[p];
        const TO cw = (TO)(TRANS ? c.wET[p] : c.wW[p]);
        const TO ce = (TO)(TRANS ? c.wWT[p] : c.wE[p]);
        const TO cs = (TO)(TRANS ? c.wNT[p] : c.wS[p]);
        const TO cn = (TO)(TRANS ? c.wST[p] : c.wN[p]);
        if (i > 1) s += cw * (TO)x[lay.addr(i - 1, j)];
        if (i < M) s += ce * (TO)x[lay.addr(i + 1, j)];
        if (j > 1) s += cs * (TO)x[lay.addr(i, j - 1)];
        if (j < M) s += cn * (TO)x[lay.addr(i, j + 1)];
        const TO v = mode ? f[p] - s : s;
        out[p] = rs ? v * (TO)rs[p] : v;   // rs = diag(A): the unscaled operator / residual
    }
}

// partial[blk*MAXV + i] = sum_k V_i[k] * w[k], i < nv <= NV (per-thread sums
// in T, block sums and everything after in FP64; deterministic order).  NV is
// the power-of-two bucket of nv, so the accumulators stay in registers; with
// VEC2 each thread reads two consecutive entries per vector (16-byte loads).
template <typename T, int NV, bool VEC2>
__global__ void __launch_bounds__(256) k_multidot(const T *__restrict__ V, long long ld, int nv,
                                                  const T *__restrict__ w, long long n, double *partials,
                                                  const int *jdev) {
    if (jdev) nv = *jdev + 1;   // captured solve: the basis size of the current iteration
    T acc[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) acc[i] = T(0);
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (VEC2) {
        typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type T2;
        const T2 *w2 = reinterpret_cast<const T2 *>(w);
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n / 2; k += stride) {
            const T2 wk = w2[k];
#pragma unroll
            for (int i = 0; i < NV; i++)
                if (i < nv) {   // two chained FMAs: on GB300 this kernel is FP64-issue-bound
                    const T2 v = reinterpret_cast<const T2 *>(V + i * ld)[k];
                    acc[i] = fma(v.x, wk.x, acc[i]);
                    acc[i] = fma(v.y, wk.y, acc[i]);
                }
        }
    } else {
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
            const T wk = w[k];
#pragma unroll
            for (int i = 0; i < NV; i++)
                if (i < nv) acc[i] += V[i * ld + k] * wk;
        }
    }
    __shared__ double sh[8][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        if (i < nv) {
            double a = (double)acc[i];
            for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(FULL, a, off);
            if (lane == 0) sh[wid][i] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q][threadIdx.x];
        partials[blockIdx.x * MAXV + threadIdx.x] = s;
    }
}

// jdev != null: nv is the largest basis size, the kernel reads the current one
template <typename T>
static void launch_multidot(blp_handle *h, int nb, const T *V, long long ld, int nv, const T *w, long long n,
                            double *partials, const int *jdev = nullptr) {
    const bool v2 = (ld % 2 == 0) && (n % 2 == 0) && ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0);
#define BLP_MD(NVB)                                                                                   \
    do {                                                                                              \
        if (v2) k_multidot<T, NVB, true><<<nb, 256, 0, h->stream>>>(V, ld, nv, w, n, partials, jdev); \
        else k_multidot<T, NVB, false><<<nb, 256, 0, h->stream>>>(V, ld, nv, w, n, partials, jdev);   \
    } while (0)
    if (nv <= 2) BLP_MD(2);
    else if (nv <= 4) BLP_MD(4);
    else if (nv <= 8) BLP_MD(8);
    else if (nv <= 16) BLP_MD(16);
    else if (nv <= 32) BLP_MD(32);
    else BLP_MD(MAXV - 1);
#undef BLP_MD
}

// out[i] = sum_b partials[b*MAXV + i] (+ add[i] if add), one warp per entry
__global__ void k_reduce(const double *partials, int nb, int nv, double *out, const double *add, const int *jdev) {
    if (jdev) nv = *jdev + 1;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < nv; i += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += partials[b * MAXV + i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(FULL, s, off);
        if (lane == 0) out[i] = s + (add ? add[i] : 0.0);
    }
}
static inline int reduce_threads(int nv) { return 32 * (nv < 32 ? nv : 32); }

// w -= sum_i V_i h_i ; optional partial sums of ||w||^2 into partials[blk*MAXV].
// NV: power-of-two bucket of nv (coefficients in registers, loop unrolled);
// VEC2: two consecutive entries per thread (16-byte loads and stores).
template <typename T, int NV, bool VEC2>
__global__ void __launch_bounds__(256) k_update(const T *__restrict__ V, long long ld, int nv, const double *__restrict__ h,
                                                T *__restrict__ w, long long n, double *partials, const int *jdev) {
    if (jdev) nv = *jdev + 1;
    T hc[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) hc[i] = i < nv ? (T)h[i] : T(0);
    T acc = T(0);
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (VEC2) {
        typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type T2;
        T2 *w2 = reinterpret_cast<T2 *>(w);
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n / 2; k += stride) {
            T2 s = w2[k];
#pragma unroll
            for (int i = 0; i < NV; i++)
                if (i < nv) {
                    const T2 v = reinterpret_cast<const T2 *>(V + i * ld)[k];
                    s.x -= v.x * hc[i];
                    s.y -= v.y * hc[i];
                }
            w2[k] = s;
            acc += s.x * s.x + s.y * s.y;
        }
    } else {
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
            T s = w[k];
#pragma unroll
            for (int i = 0; i < NV; i++)
                if (i < nv) s -= V[i * ld + k] * hc[i];
            w[k] = s;
            acc += s * s;
        }
    }
    if (partials) {
        __shared__ double sh[8];
        double a = (double)acc;
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(FULL, a, off);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
            partials[blockIdx.x * MAXV] = s;
        }
    }
}

template <typename T>
static void launch_update(blp_handle *h, int nb, const T *V, long long ld, int nv, const double *hv, T *w, long long n,
                          double *partials, const int *jdev = nullptr) {
    const bool v2 = (ld % 2 == 0) && (n % 2 == 0) && ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0);
#define BLP_UP(NVB)                                                                                   \
    do {                                                                                              \
        if (v2) k_update<T, NVB, true><<<nb, 256, 0, h->stream>>>(V, ld, nv, hv, w, n, partials, jdev); \
        else k_update<T, NVB, false><<<nb, 256, 0, h->stream>>>(V, ld, nv, hv, w, n, partials, jdev);   \
    } while (0)
    if (nv <= 2) BLP_UP(2);
    else if (nv <= 4) BLP_UP(4);
    else if (nv <= 8) BLP_UP(8);
    else if (nv <= 16) BLP_UP(16);
    else if (nv <= 32) BLP_UP(32);
    else BLP_UP(MAXV - 1);
#undef BLP_UP
}

// partial sums of ||x||^2 (and, with scale != null, of ||scale*x||^2 in slot 1)
template <typename T>
__global__ void __launch_bounds__(256) k_norm2(const T *__restrict__ x, long long n, const double *__restrict__ scale,
                                               double *partials) {
    double a = 0.0, b = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double v = (double)x[k];
        a += v * v;
        if (scale) { double u = v * scale[k]; b += u * u; }
    }
    __shared__ double sh[2][8];
    for (int off = 16; off > 0; off >>= 1) { a += __shfl_down_sync(FULL, a, off); b += __shfl_down_sync(FULL, b, off); }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = a; sh[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) { s0 += sh[0][q]; s1 += sh[1][q]; }
        partials[blockIdx.x * MAXV] = s0;
        partials[blockIdx.x * MAXV + 1] = s1;
    }
}

// y = alpha * x / s where s = *sdev (device scalar, sqrt applied if sq);
// sdev == nullptr: y = alpha * x (precision conversion)
// y = x / d elementwise (0 where d = 0: the padding slots of diag(A))
template <typename TO>
__global__ void k_div(const double *__restrict__ x, const double *__restrict__ d, TO *__restrict__ y, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double dk = d[k];
        y[k] = (TO)(dk != 0.0 ? x[k] / dk : 0.0);
    }
}

template <typename TI, typename TO>
__global__ void k_scale(const TI *__restrict__ x, TO *__restrict__ y, long long n, const double *sdev, int sq, double alpha) {
    double f = alpha;
    if (sdev) {
        double s = *sdev;
        if (sq) s = sqrt(s);
        f = s != 0.0 ? alpha / s : 0.0;
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        y[k] = (TO)((double)x[k] * f);
}

// u += alpha * sum_i Z_i y_i  (y on device, FP64)
template <typename T, typename TU>
__global__ void k_combine(const T *__restrict__ Z, long long ld, int k, const double *__restrict__ y,
                          TU *__restrict__ u, long long n, const double *alpha_dev, const int *kdev) {
    if (kdev) k = *kdev;
    __shared__ double ys[MAXV];
    const double al = alpha_dev ? *alpha_dev : 1.0;
    if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x] * al;
    __syncthreads();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; i++) s += (double)Z[i * ld + q] * ys[i];
        u[q] = (TU)((double)u[q] + s);
    }
}

// Device-side least-squares update (FP64): column j of the Hessenberg matrix
// h1 + h2 (two Gram-Schmidt passes) with subdiagonal sqrt(nrm2), previous
// Givens rotations, new rotation, residual estimate |g_{j+1}|.
struct GivensState {
    double H[MAXV * MAXV];   // H[i*MAXV + j], upper triangular after rotations
    double cs[MAXV], sn[MAXV], g[MAXV + 1], y[MAXV];
    double resid, hsub;
};
__global__ void k_givens(GivensState *G, int j, const double *h1, const double *h2, const double *nrm2,
                         const int *jdev) {
    if (threadIdx.x != 0) return;
    if (jdev) j = *jdev;
    double col[MAXV + 1];
    for (int i = 0; i <= j; i++) col[i] = h1[i] + (h2 ? h2[i] : 0.0);
    double hn = sqrt(*nrm2);
    col[j + 1] = hn;
    for (int i = 0; i < j; i++) {
        double a = col[i], b = col[i + 1];
        col[i] = G->cs[i] * a + G->sn[i] * b;
        col[i + 1] = -G->sn[i] * a + G->cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double d = sqrt(a * a + b * b);
    double c = d == 0.0 ? 1.0 : a / d, s = d == 0.0 ? 0.0 : b / d;
    G->cs[j] = c; G->sn[j] = s;
    col[j] = d;
    for (int i = 0; i <= j; i++) G->H[i * MAXV + j] = col[i];
    G->g[j + 1] = -s * G->g[j];
    G->g[j] = c * G->g[j];
    G->resid = fabs(G->g[j + 1]);
    G->hsub = hn;
}
__global__ void k_givens_init(GivensState *G, const double *beta2) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i <= MAXV; i++) G->g[i] = 0.0;
    G->g[0] = sqrt(*beta2);
    G->resid = G->g[0];
}
__global__ void k_backsolve(GivensState *G, int k, const int *kdev) {
    if (threadIdx.x != 0) return;
    if (kdev) k = *kdev;
    for (int i = k - 1; i >= 0; i--) {
        double s = G->g[i];
        for (int q = i + 1; q < k; q++) s -= G->H[i * MAXV + q] * G->y[q];
        G->y[i] = s / G->H[i * MAXV + i];
    }
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
// FGMRES work space: the basis V, the Arnoldi vector w and the solution live
// in FP64; the preconditioned vectors Z in the preconditioner's precision TZ
// (FP32 for the mixed solve, whose FP64 matrix-vector product reads them
// directly, so the Arnoldi relation holds exactly for the stored Z).
template <typename TZ>
struct KWork {
    int m;
    long long np;
    double *V, *w;
    TZ *Z;
    float *v32;        // mixed: FP32 copy of the vector being preconditioned
    double *hbuf;      // [4*MAXV]: h1, h2, norm, beta
    GivensState *G;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device control block of a captured solve (see fgmres_captured).
struct SolveCtl {
    double target;   // the FGMRES target for the normalised residual
    double res;      // residual norm at the last restart
    int fs_zero;     // zero right-hand side: nothing to solve
    int it, maxit;   // iterations so far, iteration budget
    int j, kdim;     // Arnoldi index and Krylov dimension of the current cycle
    int m, restarts;
};

struct Workspace {
    KWork<double> kd;
    KWork<float> kf;
    double *u, *f, *r, *t;    // FP64 region vectors
    void *zg;                 // captured solve: preconditioner output (either precision)
    SolveCtl *ctl;
    bool mixed;
};

static int setup_ws(blp_handle *h, Workspace &W, bool mixed) {
    const int m = h->p.restart;
    const long long np = h->lay.npad;
    size_t bytes = 0;
    auto reserve = [&](size_t b) { size_t o = bytes; bytes += align256(b); return o; };
    size_t oU = reserve(sizeof(double) * np), oF = reserve(sizeof(double) * np), oR = reserve(sizeof(double) * np),
           oT = reserve(sizeof(double) * np);
    size_t oH = reserve(sizeof(double) * 4 * MAXV), oG = reserve(sizeof(GivensState));
    size_t oV = reserve(sizeof(double) * np * (m + 2));
    size_t oZ = reserve((mixed ? sizeof(float) : sizeof(double)) * np * m);
    size_t oV32 = reserve(sizeof(float) * np);
    size_t oZG = reserve(sizeof(double) * np), oC = reserve(sizeof(SolveCtl));
    int rc = blp_internal_ensure_ws(h, bytes);
    if (rc) return rc;
    char *base = (char *)h->ws;
    CUDA_TRY(cudaMemsetAsync(base, 0, bytes, h->stream));
    W.mixed = mixed;
    W.u = (double *)(base + oU); W.f = (double *)(base + oF); W.r = (double *)(base + oR); W.t = (double *)(base + oT);
    W.zg = base + oZG;
    W.ctl = (SolveCtl *)(base + oC);
    double *hb = (double *)(base + oH);
    GivensState *G = (GivensState *)(base + oG);
    double *V = (double *)(base + oV);
    if (!mixed) W.kd = {m, np, V, V + np * (m + 1), (double *)(base + oZ), (float *)(base + oV32), hb, G};
    else W.kf = {m, np, V, V + np * (m + 1), (float *)(base + oZ), (float *)(base + oV32), hb, G};
    return BLP_OK;
}

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------
static int nblocks(long long np) { return (int)std::min<long long>(BLP_RED_BLOCKS, std::max<long long>(1, (np + 255) / 256)); }
// Blocks of the Arnoldi dot products: one per SM.  The kernel is bound by
// GB300's FP64 FMA rate (81% FP64-pipe activity under ncu), and every warp
// ends with an FP64 shuffle reduction per basis vector, so fewer warps means
// fewer FP64 instructions for the same products.
static int nblocks_dot(long long np) { return std::min(nblocks(np), 152); }


// out = Op x (mode 0) or f - Op x (mode 1); FP64 operator, x in TX precision
template <typename TX>
static int matvec(blp_handle *h, const TX *x, double *out, const double *f, int mode, int trans,
                  const double *rs = nullptr, TX *xs = nullptr, const int *jdev = nullptr) {
    long long np = h->lay.npad;
    const double nodes = (double)(h->N - 1) * (h->N - 1);
    ProfScope ps(h, KC_MATVEC, nodes * (sizeof(double) * (mode ? 6 : 5) + sizeof(TX)));   // x, 4 couplings, out (+ f)
    if (trans) k_matvec<double, TX, double, true><<<grid_for(np, 256), 256, 0, h->stream>>>(h->lay, h->cd, x, out, f, mode, rs, xs, jdev);
    else k_matvec<double, TX, double, false><<<grid_for(np, 256), 256, 0, h->stream>>>(h->lay, h->cd, x, out, f, mode, rs, xs, jdev);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

// ||x||^2 (and ||scale*x||^2) -> dst[0], dst[1] (device)
template <typename T>
static int norm2(blp_handle *h, const T *x, const double *scale, double *dst) {
    long long np = h->lay.npad;
    int nb = nblocks(np);
    { ProfScope ps_(h, KC_SMALL);
      k_norm2<T><<<nb, 256, 0, h->stream>>>(x, np, scale, h->partials);
      LAUNCH_CHECK(h); }
    { ProfScope ps_(h, KC_SMALL);
      k_reduce<<<1, 64, 0, h->stream>>>(h->partials, nb, 2, dst, nullptr, nullptr);
      LAUNCH_CHECK(h); }
    return BLP_OK;
}

static int read_doubles(blp_handle *h, const double *src, double *dst, int n) {
    CUDA_TRY(cudaMemcpyAsync(h->host_state->red, src, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < n; i++) dst[i] = h->host_state->red[i];
    return BLP_OK;
}

static int check_err(blp_handle *h) {
    int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (e) {
        CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
        return e;
    }
    return BLP_OK;
}
int blp_internal_check_err(blp_handle *h) { return check_err(h); }

// Restarted FGMRES(m) on Op x = b (Op = the normalised operator or its
// transpose) in FP64, right preconditioned by the (transposed) normalised
// preconditioner in precision TZ.  x: initial guess / result.  Stops after
// a restart whose true residual is <= target, or at maxit iterations (a
// cycle also ends early when the Arnoldi estimate reaches the target).
template <typename TZ>
// rs == nullptr: Arnoldi on the row-normalised operator D^-1 A with right-hand
// side b = D^-1 f.  rs == diag(A): Arnoldi on A itself (unscaled residuals,
// the paper's formulation), with the same b: the residual f - A x is formed
// as rs * (b - D^-1 A x), and the preconditioner, which maps v to
// (D^-1 M)^-1 v = M^-1 D v, receives D^-1 v; vs is a scratch vector.
static int fgmres(blp_handle *h, KWork<TZ> &K, const double *b, double *x, int trans, double target, int maxit,
                  int *iters, int *restarts, int *maxcyc, double *res_out, const double *rs, double *vs) {
    const long long np = K.np;
    const int m = K.m;
    int nb = nblocks(np), nbd = nblocks_dot(np);
    int it = 0;
    int rc;
    double res = 0.0;
    for (;;) {
        // r = b - Op x -> V_0
        if ((rc = matvec<double>(h, x, K.V, b, 1, trans, rs))) return rc;
        if ((rc = norm2<double>(h, K.V, nullptr, K.hbuf + 3 * MAXV))) return rc;
        double beta2;
        if ((rc = read_doubles(h, K.hbuf + 3 * MAXV, &beta2, 1))) return rc;
        res = sqrt(beta2);
        if (res <= target || it >= maxit) break;
        (*restarts)++;
        { ProfScope ps_(h, KC_SMALL);
          k_scale<double, double><<<grid_for(np, 256), 256, 0, h->stream>>>(K.V, K.V, np, K.hbuf + 3 * MAXV, 1, 1.0);
          LAUNCH_CHECK(h); }
        { ProfScope ps_(h, KC_SMALL);
          k_givens_init<<<1, 32, 0, h->stream>>>(K.G, K.hbuf + 3 * MAXV);
          LAUNCH_CHECK(h); }
        int kdim = 0;
        for (int j = 0; j < m && it < maxit; j++) {
            double *vj = K.V + j * np;
            TZ *zj = K.Z + j * np;
            int cyc = 0;
            if (sizeof(TZ) == sizeof(double)) {
                const double *vin = vj;
                if (rs) {
                    { ProfScope ps_(h, KC_SMALL);
                      k_div<double><<<grid_for(np, 256), 256, 0, h->stream>>>(vj, rs, vs, np);
                      LAUNCH_CHECK(h); }
                    vin = vs;
                }
                if ((rc = precond_apply<TZ>(h, (const TZ *)vin, zj, trans, &cyc))) return rc;
            } else {
                { ProfScope ps_(h, KC_SMALL);
                  if (rs) k_div<float><<<grid_for(np, 256), 256, 0, h->stream>>>(vj, rs, K.v32, np);
                  else k_scale<double, float><<<grid_for(np, 256), 256, 0, h->stream>>>(vj, K.v32, np, nullptr, 0, 1.0);
                  LAUNCH_CHECK(h); }
                if ((rc = precond_apply<float>(h, K.v32, (float *)zj, trans, &cyc))) return rc;
            }
            if (cyc > *maxcyc) *maxcyc = cyc;
            if ((rc = matvec<TZ>(h, zj, K.w, nullptr, 0, trans, rs))) return rc;
            // classical Gram-Schmidt, twice (mathematically the MGS step of Sec. 3.3)
            int nv = j + 1;
            double *h1 = K.hbuf, *h2 = K.hbuf + MAXV, *nr = K.hbuf + 2 * MAXV;
            { ProfScope ps_(h, KC_MULTIDOT, (double)np * sizeof(double) * (nv + 1));
              launch_multidot<double>(h, nbd, K.V, np, nv, K.w, np, h->partials);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_SMALL);
              k_reduce<<<1, reduce_threads(nv), 0, h->stream>>>(h->partials, nbd, nv, h1, nullptr, nullptr);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_UPDATE, (double)np * sizeof(double) * (nv + 2));
              launch_update<double>(h, nb, K.V, np, nv, h1, K.w, np, nullptr);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_MULTIDOT, (double)np * sizeof(double) * (nv + 1));
              launch_multidot<double>(h, nbd, K.V, np, nv, K.w, np, h->partials);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_SMALL);
              k_reduce<<<1, reduce_threads(nv), 0, h->stream>>>(h->partials, nbd, nv, h2, nullptr, nullptr);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_UPDATE, (double)np * sizeof(double) * (nv + 2));
              launch_update<double>(h, nb, K.V, np, nv, h2, K.w, np, h->partials);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_SMALL);
              k_reduce<<<1, 32, 0, h->stream>>>(h->partials, nb, 1, nr, nullptr, nullptr);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_SMALL);
              k_givens<<<1, 32, 0, h->stream>>>(K.G, j, h1, h2, nr, nullptr);
              LAUNCH_CHECK(h); }
            { ProfScope ps_(h, KC_SMALL);
              k_scale<double, double><<<grid_for(np, 256), 256, 0, h->stream>>>(K.w, K.V + (j + 1) * np, np, nr, 1, 1.0);
              LAUNCH_CHECK(h); }
            it++;
            kdim = j + 1;
            CUDA_TRY(cudaMemcpyAsync(h->host_state->red, &K.G->resid, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            const double est = h->host_state->red[0], hsub = h->host_state->red[1];
            if ((rc = check_err(h))) return rc;
            if (est <= target || hsub == 0.0) break;
        }
        { ProfScope ps_(h, KC_SMALL);
          k_backsolve<<<1, 32, 0, h->stream>>>(K.G, kdim, nullptr);
          LAUNCH_CHECK(h); }
        { ProfScope ps_(h, KC_SMALL);
          k_combine<TZ, double><<<grid_for(np, 256), 256, 0, h->stream>>>(K.Z, np, kdim, K.G->y, x, np, nullptr, nullptr);
          LAUNCH_CHECK(h); }
    }
    *iters += it;
    if (res_out) *res_out = res;
    return res <= target ? BLP_OK : BLP_ERR_NOCONV;
}

// ---------------------------------------------------------------------------
// Device-driven FGMRES: the whole restarted iteration as one CUDA graph.
//
//   WHILE (restart)                          hR: set by k_restart
//     r = b - Op x;  beta = ||r||
//     k_restart: stop (target met, budget spent, zero right-hand side, error)
//     IF (cycle)                             hC: set by k_restart
//       V_0 = r / beta;  Givens state from beta;  j = 0
//       WHILE (iterate)                      hI: set by k_cycle_start, k_iter_end
//         z = M^-1 V_j (corner cycles: a WHILE node of their own);
//         w = Op z and Z_j = z;  CGS2 against V_0..V_j;  Givens;  V_j+1 = w / h
//         k_iter_end: it++, j++; continue unless the estimate meets the
//                     target, the Arnoldi process broke down, j = m, the
//                     budget is spent or a kernel recorded an error
//       x += Z y (y from the triangular solve)
//
// The same decisions, in the same order and with the same arithmetic, as the
// host-driven loop in fgmres(); the host reads the control block once, after
// the graph.  Kernels that depend on the Arnoldi index read it from the
// control block.  The preconditioner reads and writes fixed vectors: the
// kernel that forms V_j also writes the preconditioner's input, and the
// operator kernel stores its input z into Z_j.  The graph touches only the
// handle's work space, so it is built once per handle, precision and
// direction and replayed by later solves.
// ---------------------------------------------------------------------------
__global__ void k_ctl_init(SolveCtl *c, double target, int fs_zero, int maxit, int m) {
    c->target = target;
    c->res = 0.0;
    c->fs_zero = fs_zero;
    c->it = 0;
    c->maxit = maxit;
    c->j = 0;
    c->kdim = 0;
    c->m = m;
    c->restarts = 0;
}

__global__ void k_restart(SolveCtl *c, const double *beta2, const int *err, cudaGraphConditionalHandle hR,
                          cudaGraphConditionalHandle hC) {
    const double res = sqrt(*beta2);
    c->res = res;
    const bool stop = c->fs_zero || res <= c->target || c->it >= c->maxit || *err != 0;
    if (!stop) c->restarts++;
    c->j = 0;
    c->kdim = 0;
    cudaGraphSetConditional(hR, stop ? 0u : 1u);
    cudaGraphSetConditional(hC, stop ? 0u : 1u);
}

__global__ void k_cycle_start(GivensState *G, const double *beta2, cudaGraphConditionalHandle hI) {
    for (int i = 0; i <= MAXV; i++) G->g[i] = 0.0;
    G->g[0] = sqrt(*beta2);
    G->resid = G->g[0];
    cudaGraphSetConditional(hI, 1u);
}

// V_0 = r / ||r|| in place, and the preconditioner's input (V_0 in its precision)
template <typename TO>
__global__ void k_scale_first(double *__restrict__ V, long long np, const double *beta2, TO *__restrict__ vin) {
    const double s = sqrt(*beta2);
    const double f = s != 0.0 ? 1.0 / s : 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np; k += (long long)gridDim.x * blockDim.x) {
        const double v = V[k] * f;
        V[k] = v;
        vin[k] = (TO)v;
    }
}

// V_{j+1} = w / sqrt(nrm2), and the next preconditioner input
template <typename TO>
__global__ void k_scale_col(const int *jdev, const double *__restrict__ w, double *__restrict__ V, long long np,
                            const double *nrm2, TO *__restrict__ vin) {
    const double s = sqrt(*nrm2);
    const double f = s != 0.0 ? 1.0 / s : 0.0;
    double *v = V + (long long)(*jdev + 1) * np;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np; k += (long long)gridDim.x * blockDim.x) {
        const double x = w[k] * f;
        v[k] = x;
        vin[k] = (TO)x;
    }
}

__global__ void k_iter_end(SolveCtl *c, const GivensState *G, const int *err, cudaGraphConditionalHandle hI) {
    c->it++;
    c->j++;
    c->kdim = c->j;
    const bool stop = G->resid <= c->target || G->hsub == 0.0 || c->j >= c->m || c->it >= c->maxit || *err != 0;
    cudaGraphSetConditional(hI, stop ? 0u : 1u);
}

// The preconditioner's input vector of the captured solve: the FP32 copy of
// the basis vector (mixed) or an FP64 scratch vector.
template <typename TZ>
static TZ *precond_input(Workspace &W, KWork<TZ> &K) {
    return sizeof(TZ) == 4 ? reinterpret_cast<TZ *>(K.v32) : reinterpret_cast<TZ *>(W.t);
}

// One Arnoldi step with Z_j = M^-1 V_j, j read from the control block.
template <typename TZ>
static int capture_iteration(blp_handle *h, Workspace &W, KWork<TZ> &K, int trans, cudaGraphConditionalHandle hI) {
    const long long np = K.np;
    const int m = K.m, nb = nblocks(np), nbd = nblocks_dot(np);
    const int *jdev = &W.ctl->j;
    TZ *vin = precond_input<TZ>(W, K);   // V_j, written when V_j was formed
    TZ *zg = static_cast<TZ *>(W.zg);
    double *h1 = K.hbuf, *h2 = K.hbuf + MAXV, *nr = K.hbuf + 2 * MAXV;
    int rc, cyc = 0;
    if ((rc = precond_apply<TZ>(h, vin, zg, trans, &cyc))) return rc;
    if ((rc = matvec<TZ>(h, zg, K.w, nullptr, 0, trans, nullptr, K.Z, jdev))) return rc;   // and Z_j = z
    launch_multidot<double>(h, nbd, K.V, np, m, K.w, np, h->partials, jdev);
    LAUNCH_CHECK(h);
    k_reduce<<<1, reduce_threads(m), 0, h->stream>>>(h->partials, nbd, m, h1, nullptr, jdev);
    LAUNCH_CHECK(h);
    launch_update<double>(h, nb, K.V, np, m, h1, K.w, np, nullptr, jdev);
    LAUNCH_CHECK(h);
    launch_multidot<double>(h, nbd, K.V, np, m, K.w, np, h->partials, jdev);
    LAUNCH_CHECK(h);
    k_reduce<<<1, reduce_threads(m), 0, h->stream>>>(h->partials, nbd, m, h2, nullptr, jdev);
    LAUNCH_CHECK(h);
    launch_update<double>(h, nb, K.V, np, m, h2, K.w, np, h->partials, jdev);
    LAUNCH_CHECK(h);
    k_reduce<<<1, 32, 0, h->stream>>>(h->partials, nb, 1, nr, nullptr, nullptr);
    LAUNCH_CHECK(h);
    k_givens<<<1, 32, 0, h->stream>>>(K.G, 0, h1, h2, nr, jdev);
    LAUNCH_CHECK(h);
    k_scale_col<TZ><<<grid_for(np, 256), 256, 0, h->stream>>>(jdev, K.w, K.V, np, nr, vin);
    LAUNCH_CHECK(h);
    k_iter_end<<<1, 1, 0, h->stream>>>(W.ctl, K.G, h->err, hI);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

struct CapturedCounts { long long restart, cycle, iter; };

template <typename TZ>
static int capture_solve(blp_handle *h, Workspace &W, KWork<TZ> &K, int trans, CapturedCounts *cnt) {
    const long long np = K.np;
    int rc;
    cudaGraphConditionalHandle hR, hC, hI;
    const long long l0 = h->launches;
    if ((rc = cap_handle(h, 1, &hR))) return rc;
    if ((rc = cap_begin(h, hR, cudaGraphCondTypeWhile))) return rc;
    {
        const long long l1 = h->launches;
        if ((rc = matvec<double>(h, W.u, K.V, W.f, 1, trans))) return rc;
        if ((rc = norm2<double>(h, K.V, nullptr, K.hbuf + 3 * MAXV))) return rc;
        if ((rc = cap_handle(h, 0, &hC))) return rc;
        k_restart<<<1, 1, 0, h->stream>>>(W.ctl, K.hbuf + 3 * MAXV, h->err, hR, hC);
        LAUNCH_CHECK(h);
        cnt->restart = h->launches - l1;
        if ((rc = cap_begin(h, hC, cudaGraphCondTypeIf))) return rc;
        {
            const long long l2 = h->launches;
            k_scale_first<TZ><<<grid_for(np, 256), 256, 0, h->stream>>>(K.V, np, K.hbuf + 3 * MAXV, precond_input<TZ>(W, K));
            LAUNCH_CHECK(h);
            if ((rc = cap_handle(h, 0, &hI))) return rc;
            k_cycle_start<<<1, 1, 0, h->stream>>>(K.G, K.hbuf + 3 * MAXV, hI);
            LAUNCH_CHECK(h);
            if ((rc = cap_begin(h, hI, cudaGraphCondTypeWhile))) return rc;
            const long long l3 = h->launches;
            rc = capture_iteration<TZ>(h, W, K, trans, hI);
            cnt->iter = h->launches - l3;
            if (rc) return rc;
            if ((rc = cap_end(h))) return rc;
            k_backsolve<<<1, 32, 0, h->stream>>>(K.G, 0, &W.ctl->kdim);
            LAUNCH_CHECK(h);
            k_combine<TZ, double><<<grid_for(np, 256), 256, 0, h->stream>>>(K.Z, np, 0, K.G->y, W.u, np, nullptr,
                                                                           &W.ctl->kdim);
            LAUNCH_CHECK(h);
            cnt->cycle = h->launches - l2 - cnt->iter;
        }
        if ((rc = cap_end(h))) return rc;
    }
    if ((rc = cap_end(h))) return rc;
    h->launches = l0;   // counted when the graph runs
    return BLP_OK;
}

static_assert(sizeof(SolveCtl) <= sizeof(DevState::red), "the control block is read back through host_state->red");

// Run the captured solve (building its graph on first use).  Adds the
// iterations and restarts the device took; the caller forms the residuals.
// *fallback is set when the graph cannot be built (nothing was launched):
// the caller then runs the host-driven loop instead.
template <typename TZ>
static int fgmres_captured(blp_handle *h, Workspace &W, KWork<TZ> &K, int trans, double target, bool fs_zero,
                           int maxit, int *iters, int *restarts, bool *fallback) {
    *fallback = false;
    const int prec = sizeof(TZ) == 4 ? 1 : 0;
    blp_handle::SolveGraph &SG = h->solve_graph[prec][trans ? 1 : 0];
    if (SG.exec && (SG.ws != h->ws || SG.m != K.m)) {
        cudaGraphExecDestroy(SG.exec);
        SG.exec = nullptr;
    }
    if (!SG.exec) {
        *fallback = true;
        int rc = precond_capture_prepare<TZ>(h);
        if (rc) return rc;
        for (int q = 0; q < 4; q++)
            if (!h->cap[q]) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap[q], cudaStreamNonBlocking));
        CapturedCounts cnt = {0, 0, 0};
        h->corner_body_launches = 0;
        CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        rc = capture_solve<TZ>(h, W, K, trans, &cnt);
        h->capturing = false;
        if (rc) {
            cap_abort(h);
            return rc;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&SG.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            SG.exec = nullptr;
            return BLP_ERR_CUDA;
        }
        SG.ws = h->ws;
        SG.m = K.m;
        SG.n_restart = cnt.restart;
        SG.n_cycle = cnt.cycle;
        SG.n_iter = cnt.iter;
        SG.n_corner = h->corner_body_launches;
        *fallback = false;
    }
    k_ctl_init<<<1, 1, 0, h->stream>>>(W.ctl, target, fs_zero ? 1 : 0, maxit, K.m);
    LAUNCH_CHECK(h);
    CUDA_TRY(cudaGraphLaunch(SG.exec, h->stream));
    SolveCtl c;
    CUDA_TRY(cudaMemcpyAsync(h->host_state->red, W.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(&h->host_state->flags[4], &h->dev->flags[4], sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    memcpy(&c, h->host_state->red, sizeof(SolveCtl));
    *iters += c.it;
    *restarts += c.restarts;
    // kernels the graph ran: one restart body per restart plus the final
    // check, one cycle body per restart, one iteration body per iteration,
    // and the corner cycles beyond the first of each application
    const long long extra_cycles = std::max(0LL, (long long)h->host_state->flags[4] - c.it);
    h->launches += SG.n_restart * (c.restarts + 1) + SG.n_cycle * c.restarts + SG.n_iter * c.it + SG.n_corner * extra_cycles;
    return BLP_OK;
}

// ---------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------
static bool is_dev(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// stage a caller array (host or device) of n doubles into device memory
static int stage_in(blp_handle *h, const double *src, int slot, const double **dst) {
    if (is_dev(src)) { *dst = src; return BLP_OK; }
    long long n = (long long)(h->N - 1) * (h->N - 1);
    CUDA_TRY(cudaMemcpyAsync(h->stage[slot], src, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    *dst = h->stage[slot];
    return BLP_OK;
}

// the forward (trans = 0) or adjoint (trans = 1) solve, FP64 or mixed
static int solve_common(blp_handle *h, const double *f_in, double *u_io, double tol, blp_info *info, int trans) {
    auto t0 = std::chrono::steady_clock::now();
    if (!h || !f_in || !u_io || !(tol > 0.0)) return BLP_ERR_ARG;
    const long long n = (long long)(h->N - 1) * (h->N - 1);
    const bool mixed = h->p.precision == BLP_MIXED;
    Workspace W;
    int rc = setup_ws(h, W, mixed);
    if (rc) return rc;
    const double *f_dev, *u_dev_in;
    if ((rc = stage_in(h, f_in, 0, &f_dev))) return rc;
    bool u_is_dev = is_dev(u_io);
    if ((rc = stage_in(h, u_io, 1, &u_dev_in))) return rc;
    // normalised system: forward D^-1 A u = D^-1 f; adjoint (D^-1 A)^T mu = g, mu = D lambda
    if ((rc = blp_internal_to_region(h, f_dev, W.f, trans ? 0 : 1))) return rc;
    if ((rc = blp_internal_to_region(h, u_dev_in, W.u, trans ? 2 : 0))) return rc;

    // norms of the right-hand side: scaled (slot 0) and unscaled (slot 1)
    double *nb_dev = h->partials + BLP_SCALARS_OFF;   // scalars after the partial sums
    if ((rc = norm2<double>(h, W.f, trans ? nullptr : h->aC, nb_dev))) return rc;
    double fn2[2];
    if ((rc = read_doubles(h, nb_dev, fn2, 2))) return rc;
    double fs = sqrt(fn2[0]), fu = trans ? fs : sqrt(fn2[1]);
    const int mode = h->p.stop_mode;
    // target for the normalised residual
    double target_scaled = mode == BLP_STOP_SCALED ? tol * fs : 0.0;
    double target_unscaled = mode == BLP_STOP_REL2 ? tol * fu : (mode == BLP_STOP_ABS2 ? tol : 0.0);

    int iters = 0, restarts = 0, maxcyc = 0, status = BLP_ERR_NOCONV, device_driven = 0;
    double res_s = 0.0, res_u = 0.0;
    // true residuals of the current u in both norms
    auto true_res = [&](double &rs, double &ru) -> int {
        int r2 = matvec<double>(h, W.u, W.r, W.f, 1, trans);
        if (r2) return r2;
        r2 = norm2<double>(h, W.r, trans ? nullptr : h->aC, nb_dev);
        if (r2) return r2;
        double v[2];
        r2 = read_doubles(h, nb_dev, v, 2);
        rs = sqrt(v[0]);
        ru = trans ? rs : sqrt(v[1]);
        return r2;
    };
    auto met = [&](double rs, double ru) {
        return mode == BLP_STOP_SCALED ? rs <= target_scaled : ru <= target_unscaled;
    };
    CUDA_TRY(cudaMemsetAsync(&h->dev->flags[3], 0, 2 * sizeof(int), h->stream));   // flags[3], flags[4]
    if ((rc = true_res(res_s, res_u))) return rc;
    if (fs == 0.0) {
        status = BLP_OK;
    } else {
        const int budget = h->p.maxit;
        // in FP64 the unscaled stopping rules run Arnoldi on A itself, so that
        // FGMRES minimises the residual in the norm it stops on (the paper's
        // formulation, Sec. 3.3).  The scaled rule, the adjoint and the mixed
        // path use D^-1 A: an FP32 preconditioner fed D^-1 v for unscaled v
        // (entries spanning the diagonal's ~1e11 range) loses the layer rows.
        const double *rs = (!trans && !mixed && mode != BLP_STOP_SCALED) ? h->aC : nullptr;
        // device-driven iteration (one graph launch) under the scaled rule
        bool host_loop = true;
        if (h->solve_graphs && h->use_graphs && h->stream != 0 && !h->prof.on && mode == BLP_STOP_SCALED &&
            !met(res_s, res_u)) {
            bool fallback = false;
            if (mixed) rc = fgmres_captured<float>(h, W, W.kf, trans, target_scaled, false, budget, &iters, &restarts, &fallback);
            else rc = fgmres_captured<double>(h, W, W.kd, trans, target_scaled, false, budget, &iters, &restarts, &fallback);
            if (fallback) {
                h->solve_graphs = false;   // this handle keeps the host-driven loop
            } else {
                if (rc) return rc;
                if ((rc = true_res(res_s, res_u))) return rc;
                host_loop = false;
                device_driven = 1;
                // the host-driven loop counts fixed corner cycles on the host
                if (h->p.corner_fixed_cycles > 0 && iters > 0) maxcyc = std::max(maxcyc, h->p.corner_fixed_cycles);
            }
        }
        while (host_loop && !met(res_s, res_u) && iters < budget) {
            // without rs the Arnoldi estimate tracks the normalised residual:
            // for the unscaled rules convert the target with the current ratio
            double tgt = mode == BLP_STOP_SCALED ? target_scaled
                                                 : (rs ? target_unscaled : target_unscaled * (res_s / std::max(res_u, 1e-300)));
            double dummy;
            int it0 = iters;
            if (mixed) rc = fgmres<float>(h, W.kf, W.f, W.u, trans, tgt, budget - iters, &iters, &restarts, &maxcyc, &dummy, rs, W.t);
            else rc = fgmres<double>(h, W.kd, W.f, W.u, trans, tgt, budget - iters, &iters, &restarts, &maxcyc, &dummy, rs, W.t);
            if (rc != BLP_OK && rc != BLP_ERR_NOCONV) return rc;
            if ((rc = true_res(res_s, res_u))) return rc;
            if (iters == it0) break;
        }
        status = met(res_s, res_u) ? BLP_OK : BLP_ERR_NOCONV;
    }
    // write back
    double *u_out_dev = u_is_dev ? u_io : h->stage[1];
    if ((rc = blp_internal_from_region(h, W.u, u_out_dev, trans ? 1 : 0))) return rc;
    if (!u_is_dev)
        CUDA_TRY(cudaMemcpyAsync(u_io, u_out_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    int e = check_err(h);
    if (e) status = e;
    {
        int devmax = 0;
        CUDA_TRY(cudaMemcpyAsync(&devmax, &h->dev->flags[3], sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (devmax > maxcyc) maxcyc = devmax;
    }
    if (info) {
        info->status = status;
        info->iters = iters;
        info->restarts = restarts;
        info->corner_cycles_max = maxcyc;
        info->relres = mode == BLP_STOP_SCALED ? (fs > 0 ? res_s / fs : 0.0)
                                               : (mode == BLP_STOP_REL2 ? (fu > 0 ? res_u / fu : 0.0) : res_u);
        info->relres_unscaled = fu > 0 ? res_u / fu : 0.0;
        info->t_setup_ms = h->t_setup_ms;
        info->device_driven = device_driven;
        info->t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

// The legacy default stream cannot be captured into graphs: a solve issued
// on it runs on a private non-blocking stream of the handle instead, ordered
// after the caller's earlier work by an event.  The call returns after the
// work has completed, as on any other stream.
static int solve_on_capturable_stream(blp_handle *h, const double *f, double *u, double tol, blp_info *info, int trans) {
    if (!h) return BLP_ERR_ARG;
    if (h->stream != 0 || !h->use_graphs) return solve_common(h, f, u, tol, info, trans);
    if (!h->own_stream) {
        if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            h->own_stream = nullptr;
            return solve_common(h, f, u, tol, info, trans);
        }
    }
    cudaEvent_t ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->own_stream, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return BLP_ERR_CUDA;
    h->stream = h->own_stream;
    int rc = solve_common(h, f, u, tol, info, trans);
    cudaStreamSynchronize(h->own_stream);
    h->stream = 0;
    return rc;
}

extern "C" int blp_solve(blp_handle *h, const double *f, double *u, double tol, blp_info *info) {
    return solve_on_capturable_stream(h, f, u, tol, info, 0);
}
extern "C" int blp_solve_adjoint(blp_handle *h, const double *g, double *lambda, double tol, blp_info *info) {
    if (h && h->semi) return BLP_ERR_ARG;   // the parabolic-layer corner cycle is forward only
    return solve_on_capturable_stream(h, g, lambda, tol, info, 1);
}

// ---------------------------------------------------------------------------
// operator / preconditioner access and the gradient
// ---------------------------------------------------------------------------
__global__ void k_grad(int N, const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ u,
                       const double *__restrict__ lam, double *g1, double *g2, double *gr) {
    const int M = N - 1;
    long long n = (long long)M * M;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % M) + 1, j = (int)(k / M) + 1;
        const double uk = u[k], lk = lam[k];
        const double uE = i < M ? u[k + 1] : 0.0, uN = j < M ? u[k + M] : 0.0;
        if (g1) g1[k] = -lk * (uk - uE) / (x[i + 1] - x[i]);
        if (g2) g2[k] = -lk * (uk - uN) / (y[j + 1] - y[j]);
        if (gr) gr[k] = -lk * uk;
    }
}

extern "C" int blp_grad(blp_handle *h, const double *u, const double *lambda, double *g_c1, double *g_c2, double *g_r) {
    if (!h || !u || !lambda) return BLP_ERR_ARG;
    const long long n = (long long)(h->N - 1) * (h->N - 1);
    const double *ud, *ld;
    int rc;
    if ((rc = stage_in(h, u, 0, &ud))) return rc;
    if ((rc = stage_in(h, lambda, 1, &ld))) return rc;
    double *outs[3] = {g_c1, g_c2, g_r}, *dev[3];
    bool host[3];
    for (int q = 0; q < 3; q++) {
        host[q] = outs[q] && !is_dev(outs[q]);
        dev[q] = outs[q] ? (host[q] ? nullptr : outs[q]) : nullptr;
    }
    // host outputs go through the remaining staging buffers, one at a time
    for (int q = 0; q < 3; q++) {
        double *d = dev[q];
        if (host[q]) d = h->stage[2 + (q == 2 ? 1 : 0)];
        if (!outs[q]) continue;
        k_grad<<<grid_for(n, 256), 256, 0, h->stream>>>(h->N, h->x, h->y, ud, ld, q == 0 ? d : nullptr, q == 1 ? d : nullptr,
                                                       q == 2 ? d : nullptr);
        LAUNCH_CHECK(h);
        if (host[q]) CUDA_TRY(cudaMemcpyAsync(outs[q], d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    return BLP_OK;
}

extern "C" int blp_apply_operator(blp_handle *h, const double *u, double *y, int transpose) {
    if (!h || !u || !y) return BLP_ERR_ARG;
    const long long n = (long long)(h->N - 1) * (h->N - 1);
    Workspace W;
    int rc = setup_ws(h, W, false);
    if (rc) return rc;
    const double *ud;
    if ((rc = stage_in(h, u, 0, &ud))) return rc;
    // A u = D (D^-1 A) u ;  A^T u = (D^-1 A)^T (D u)
    if ((rc = blp_internal_to_region(h, ud, W.u, transpose ? 2 : 0))) return rc;
    if ((rc = matvec<double>(h, W.u, W.r, nullptr, 0, transpose))) return rc;
    bool ydev = is_dev(y);
    double *yd = ydev ? y : h->stage[2];
    if ((rc = blp_internal_from_region(h, W.r, yd, transpose ? 0 : 2))) return rc;
    if (!ydev) CUDA_TRY(cudaMemcpyAsync(y, yd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return BLP_OK;
}

extern "C" int blp_precond_apply(blp_handle *h, const double *v, double *z, int transpose, int precision, int *cycles) {
    if (!h || !v || !z) return BLP_ERR_ARG;
    const long long n = (long long)(h->N - 1) * (h->N - 1);
    const long long np = h->lay.npad;
    Workspace W;
    int rc = setup_ws(h, W, precision == BLP_MIXED);
    if (rc) return rc;
    const double *vd;
    if ((rc = stage_in(h, v, 0, &vd))) return rc;
    if ((rc = blp_internal_to_region(h, vd, W.u, 0))) return rc;
    int cyc = 0;
    if (precision == BLP_MIXED) {
        float *v32 = W.kf.v32, *z32 = W.kf.Z;
        { ProfScope ps_(h, KC_SMALL);
          k_scale<double, float><<<grid_for(np, 256), 256, 0, h->stream>>>(W.u, v32, np, nullptr, 0, 1.0);
          LAUNCH_CHECK(h); }
        if ((rc = precond_apply<float>(h, v32, z32, transpose, &cyc))) return rc;
        { ProfScope ps_(h, KC_SMALL);
          k_scale<float, double><<<grid_for(np, 256), 256, 0, h->stream>>>(z32, W.r, np, nullptr, 0, 1.0);
          LAUNCH_CHECK(h); }
    } else {
        if ((rc = precond_apply<double>(h, W.u, W.r, transpose, &cyc))) return rc;
    }
    if (cyc < 0) {   // counted on the device by the fused corner kernel
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        CUDA_TRY(cudaMemcpyAsync(&cyc, &h->dev->flags[1], sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    bool zdev = is_dev(z);
    double *zd = zdev ? z : h->stage[2];
    if ((rc = blp_internal_from_region(h, W.r, zd, 0))) return rc;
    if (!zdev) CUDA_TRY(cudaMemcpyAsync(z, zd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if ((rc = check_err(h))) return rc;
    if (cycles) *cycles = cyc;
    return BLP_OK;
}
