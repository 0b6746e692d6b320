// blp_1d.cu -- the one-dimensional method of Sec. 2, batched on the GPU.
//
// Each problem is -eps u'' - c(x) u' + r(x) u = f on (0,1), u(0) = u(1) = 0
// (eq. 1D), discretised by the upwind scheme of eq. (stencil_1d) on the
// Shishkin mesh of eq. (tau 1D) (q = 1/2: N/2 intervals on [0, tau]), and
// solved by GMRES without restarts on the left-preconditioned system
// M^-1 A u = M^-1 f, M of eq. (block_M), stopping on the true residual
// ||f - A u||_inf (Sec. 2.5.1).  Left preconditioning is the setting of the
// paper's Table 2 (MATLAB's gmres preconditions on the left).
//
// A 1D problem is a tridiagonal system of at most a few thousand unknowns:
// far too small to spread over the GPU.  The batch is what fills it: one
// thread runs one whole problem serially (assembly, preconditioner factors,
// Arnoldi with modified Gram-Schmidt, Givens rotations, the true-residual
// test), with its vectors in a private slice of one workspace, and the
// problems of the batch run side by side on every SM.
#include "blp_common.cuh"

#include <vector>

namespace {

// M of eq. (block_M) keeps A on the layer block L (unknowns 0..NL-1, nodes
// 1..NL) and both coupling entries, and the upper triangle of the interior
// block I: the interior rows q >= NL+1 lose their sub-diagonal entry.  So
// M z = v is solved by back substitution over the interior rows, then a
// Thomas solve over rows 0..NL with z_{NL+1} moved to the right-hand side.
struct Tri1D {
    int n, NL;
    const double *sub, *dia, *sup;
    const double *cp, *rp;   // Thomas factors of rows 0..NL: c'_q and 1 / pivot_q

    __device__ void precond(const double *v, double *z) const {
        z[n - 1] = v[n - 1] / dia[n - 1];
        for (int q = n - 2; q > NL; q--) z[q] = (v[q] - sup[q] * z[q + 1]) / dia[q];
        z[0] = v[0] * rp[0];
        for (int q = 1; q < NL; q++) z[q] = (v[q] - sub[q] * z[q - 1]) * rp[q];
        z[NL] = (v[NL] - sup[NL] * z[NL + 1] - sub[NL] * z[NL - 1]) * rp[NL];
        for (int q = NL - 1; q >= 0; q--) z[q] = z[q] - cp[q] * z[q + 1];
    }
    __device__ void matvec(const double *z, double *w) const {
        w[0] = dia[0] * z[0] + sup[0] * z[1];
        for (int q = 1; q < n - 1; q++) w[q] = sub[q] * z[q - 1] + dia[q] * z[q] + sup[q] * z[q + 1];
        w[n - 1] = sub[n - 1] * z[n - 2] + dia[n - 1] * z[n - 1];
    }
};

__device__ double dot(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int q = 0; q < n; q++) s += a[q] * b[q];
    return s;
}

// words of workspace per problem (kept in step with the carve-up in k_gmres_1d)
__host__ __device__ long long ws_words(int N, int m) {
    const long long n = N - 1;
    const long long w = (m + 10LL) * n + (m + 1LL) * m + 4LL * m + 8;
    return (w + 31) & ~31LL;
}

__global__ void k_gmres_1d(blp_1d_problem *P, const long long *off, double *ws, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    blp_1d_problem &p = P[k];
    const int N = p.N, n = N - 1, NL = N / 2, m = p.maxit;
    double *W = ws + off[k];
    double *sub = W, *dia = sub + n, *sup = dia + n, *cp = sup + n, *rp = cp + n;
    double *z = rp + n, *w = z + n, *t = w + n, *x = t + n, *V = x + n;
    double *H = V + (long long)(m + 1) * n;              // (m+1) x m, column j at H + j (m+1)
    double *cs = H + (long long)(m + 1) * m, *sn = cs + m, *g = sn + m, *y = g + m + 1;

    // mesh, eq. (tau 1D) with q = 1/2
    double tau = p.sigma * p.eps * log((double)N) / p.c_low;
    if (tau > 0.5) tau = 0.5;
    auto node = [&](int i) -> double {
        if (i <= NL) return ((double)i / (double)NL) * tau;
        if (i >= N) return 1.0;
        return tau + ((double)(i - NL) / (double)(N - NL)) * (1.0 - tau);
    };
    // upwind stencil, eq. (stencil_1d): unknown q is node q+1
    for (int q = 0; q < n; q++) {
        const double xm = node(q), x0 = node(q + 1), xp = node(q + 2);
        const double hi = x0 - xm, hi1 = xp - x0, hb = 0.5 * (hi + hi1);
        const double ci = p.c[q], ri = p.r[q];
        sub[q] = -p.eps / (hi * hb);
        dia[q] = p.eps / hb * (1.0 / hi + 1.0 / hi1) + ci / hi1 + ri;
        sup[q] = -p.eps / (hi1 * hb) - ci / hi1;
    }
    // Thomas factors of M's rows 0..NL (row NL's super-diagonal entry goes to
    // the right-hand side, so c'_NL is not needed)
    rp[0] = 1.0 / dia[0];
    cp[0] = sup[0] * rp[0];
    for (int q = 1; q <= NL; q++) {
        rp[q] = 1.0 / (dia[q] - sub[q] * cp[q - 1]);
        cp[q] = q < NL ? sup[q] * rp[q] : 0.0;
    }
    const Tri1D A{n, NL, sub, dia, sup, cp, rp};

    // GMRES from u = 0 on M^-1 A u = M^-1 f: the true residual of u = 0 is f,
    // the Krylov space starts at M^-1 f
    double beta = 0.0, res = 0.0;
    for (int q = 0; q < n; q++) {
        res = fmax(res, fabs(p.f[q]));
        x[q] = 0.0;
    }
    int it = 0, status = BLP_ERR_NOCONV;
    if (res <= p.stop) {
        status = BLP_OK;
    } else {
        A.precond(p.f, z);
        beta = sqrt(dot(z, z, n));
        for (int q = 0; q < n; q++) V[q] = z[q] / beta;
        g[0] = beta;
        for (int j = 0; j < m; j++) {
            double *Hj = H + (long long)j * (m + 1);
            A.matvec(V + (long long)j * n, t);
            A.precond(t, w);
            for (int i = 0; i <= j; i++) {   // modified Gram-Schmidt
                const double *Vi = V + (long long)i * n;
                const double hij = dot(w, Vi, n);
                Hj[i] = hij;
                for (int q = 0; q < n; q++) w[q] -= hij * Vi[q];
            }
            const double hn = sqrt(dot(w, w, n));
            Hj[j + 1] = hn;
            if (hn > 0.0) {
                double *Vn = V + (long long)(j + 1) * n;
                for (int q = 0; q < n; q++) Vn[q] = w[q] / hn;
            }
            // least squares min ||beta e1 - H y|| by Givens rotations
            for (int i = 0; i < j; i++) {
                const double a = Hj[i], b = Hj[i + 1];
                Hj[i] = cs[i] * a + sn[i] * b;
                Hj[i + 1] = -sn[i] * a + cs[i] * b;
            }
            const double a = Hj[j], b = Hj[j + 1], rr = sqrt(a * a + b * b);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? b / rr : 0.0;
            Hj[j] = rr;
            Hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = j; i >= 0; i--) {
                double s = g[i];
                for (int l = i + 1; l <= j; l++) s -= H[(long long)l * (m + 1) + i] * y[l];
                y[i] = H[(long long)i * (m + 1) + i] != 0.0 ? s / H[(long long)i * (m + 1) + i] : 0.0;
            }
            // iterate u = V y and its true residual (the stopping rule of Sec. 2.5.1)
            for (int q = 0; q < n; q++) x[q] = 0.0;
            for (int i = 0; i <= j; i++) {
                const double *Vi = V + (long long)i * n;
                for (int q = 0; q < n; q++) x[q] += y[i] * Vi[q];
            }
            A.matvec(x, w);
            res = 0.0;
            for (int q = 0; q < n; q++) res = fmax(res, fabs(p.f[q] - w[q]));
            it = j + 1;
            if (res <= p.stop || hn == 0.0) {
                status = BLP_OK;
                break;
            }
        }
    }
    for (int q = 0; q < n; q++) p.u[q] = x[q];
    p.iters = it;
    p.resid = res;
    p.status = status;
}

bool device_array(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int blp_solve_1d_batched(blp_1d_problem *probs, int count, void *stream) {
    if (count < 0 || (count > 0 && !probs)) return BLP_ERR_ARG;
    if (count == 0) return BLP_OK;
    std::vector<long long> off(count);
    long long total = 0;
    int bad = BLP_OK;
    for (int k = 0; k < count; k++) {
        blp_1d_problem &p = probs[k];
        p.iters = 0;
        p.resid = -1.0;
        const bool ok = p.N >= 8 && p.N <= BLP_1D_MAX_N && !(p.N & 1) && p.eps > 0.0 && p.eps <= 1.0 &&
                        p.c_low > 0.0 && p.sigma > 0.0 && p.maxit >= 1 && p.maxit <= BLP_1D_MAXIT && p.stop >= 0.0 &&
                        device_array(p.c) && device_array(p.r) && device_array(p.f) && device_array(p.u);
        p.status = ok ? -1 : BLP_ERR_ARG;
        if (!ok) {
            if (bad == BLP_OK) bad = BLP_ERR_ARG;
            continue;
        }
        off[k] = total;
        total += ws_words(p.N, p.maxit);
    }
    if (bad != BLP_OK) return bad;   // nothing runs unless every problem is valid
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *ws = nullptr;
    long long *doff = nullptr;
    blp_1d_problem *dp = nullptr;
    int rc = BLP_OK;
    if (cudaMallocAsync((void **)&ws, sizeof(double) * total, s) != cudaSuccess ||
        cudaMallocAsync((void **)&doff, sizeof(long long) * count, s) != cudaSuccess ||
        cudaMallocAsync((void **)&dp, sizeof(blp_1d_problem) * count, s) != cudaSuccess)
        rc = BLP_ERR_MEM;
    std::vector<blp_1d_problem> back(count);
    if (rc == BLP_OK && (cudaMemcpyAsync(doff, off.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                         cudaMemcpyAsync(dp, probs, sizeof(blp_1d_problem) * count, cudaMemcpyHostToDevice, s) != cudaSuccess))
        rc = BLP_ERR_CUDA;
    if (rc == BLP_OK) {
        k_gmres_1d<<<(count + 63) / 64, 64, 0, s>>>(dp, doff, ws, count);
        if (cudaGetLastError() != cudaSuccess) rc = BLP_ERR_CUDA;
    }
    if (rc == BLP_OK &&
        cudaMemcpyAsync(back.data(), dp, sizeof(blp_1d_problem) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = BLP_ERR_CUDA;
    if (ws) cudaFreeAsync(ws, s);
    if (doff) cudaFreeAsync(doff, s);
    if (dp) cudaFreeAsync(dp, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = BLP_ERR_CUDA;
    if (rc != BLP_OK) {
        cudaGetLastError();
        return rc;
    }
    int first = BLP_OK;
    for (int k = 0; k < count; k++) {
        probs[k].iters = back[k].iters;
        probs[k].resid = back[k].resid;
        probs[k].status = back[k].status;
        if (first == BLP_OK && back[k].status != BLP_OK) first = back[k].status;
    }
    return first;
}
