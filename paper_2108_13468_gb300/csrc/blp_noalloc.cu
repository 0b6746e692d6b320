// blp_noalloc.cu -- residual and residual norms of the assembled operator
// without any allocation and without a solver handle.
//
// Who needs it: a caller that must check a solution but cannot allocate
// device memory at that point -- a process whose device memory is already
// reserved (by a caching allocator or by other solver handles), a code path
// where the implicit device-wide synchronisation of cudaMalloc/cudaFree
// would stall other streams, or a monitor that verifies solutions produced
// elsewhere and holds no blp_handle (whose workspace is allocated by
// blp_setup).  This call uses only the caller's arrays and a fixed
// file-scope device array for its reduction partials.
//
// The operator is the same upwind 5-point stencil that blp_setup assembles;
// the two paths share no code, so their results agree to rounding only.

#include <cuda_runtime.h>

#include "../../include/blp.h"

namespace {

// Scratch layout (doubles): [0] completion ticket (low 32 bits, as an
// unsigned int), [1..4] the four norms, [kRows + 4*(j-1) + q] the partial
// sums q = 0..3 of grid row j.  Rows are written before they are read in
// every call; only the ticket must start at zero, and each call clears it.
constexpr int kRows = 8;
constexpr int kScratchDoubles = kRows + 4 * BLP_NOALLOC_MAX_N;  // 256 KiB + 64 B
constexpr int kThreads = 256;

static __device__ __align__(256) double blp_noalloc_scratch[kScratchDoubles];

// Deterministic block sum of four values (fixed shuffle tree, then warps in
// index order); the result is valid in thread 0.
__device__ void block_sum4(double v[4]) {
    __shared__ double part[kThreads / 32][4];
    for (int q = 0; q < 4; q++)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < 4; q++) part[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; q++) {
            double s = 0.0;
            for (int k = 0; k < kThreads / 32; k++) s += part[k][q];
            v[q] = s;
        }
    }
    __syncthreads();
}

// One CTA per grid row j.  Residual s = f - A u with the Sec. 3 stencil
// assembled on the fly from the mesh and the coefficient fields; row partial
// sums of s^2, (s/aC)^2, f^2, (f/aC)^2 go to the scratch; the CTA that
// finishes last sums the rows in index order (the same order whichever CTA
// that is) and writes the four norms.
__global__ void __launch_bounds__(kThreads) k_residual_noalloc(int N, const double *__restrict__ x,
                                                               const double *__restrict__ y, double eps,
                                                               const double *__restrict__ c1,
                                                               const double *__restrict__ c2,
                                                               const double *__restrict__ r,
                                                               const double *__restrict__ f,
                                                               const double *__restrict__ u, double *__restrict__ res,
                                                               double *scratch) {
    const int n1 = N - 1;
    const int j = blockIdx.x + 1;
    const double kj = y[j] - y[j - 1], kj1 = y[j + 1] - y[j];
    const double kb = 0.5 * (kj + kj1);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x + 1; i <= n1; i += kThreads) {
        const long long k = (long long)(j - 1) * n1 + (i - 1);
        const double hi = x[i] - x[i - 1], hi1 = x[i + 1] - x[i];
        const double hb = 0.5 * (hi + hi1);
        const double C1 = c1[k], C2 = c2[k], R = r[k];
        const double aW = -eps / (hb * hi);
        const double aE = -eps / (hb * hi1) - C1 / hi1;
        const double aS = -eps / (kb * kj);
        const double aN = -eps / (kb * kj1) - C2 / kj1;
        const double aC = eps / hb * (1.0 / hi + 1.0 / hi1) + eps / kb * (1.0 / kj + 1.0 / kj1) + C1 / hi1 + C2 / kj1 + R;
        double Au = aC * u[k];
        if (i > 1) Au += aW * u[k - 1];
        if (i < n1) Au += aE * u[k + 1];
        if (j > 1) Au += aS * u[k - n1];
        if (j < n1) Au += aN * u[k + n1];
        const double fk = f[k], s = fk - Au;
        if (res) res[k] = s;
        const double sd = s / aC, fd = fk / aC;
        acc[0] += s * s;
        acc[1] += sd * sd;
        acc[2] += fk * fk;
        acc[3] += fd * fd;
    }
    block_sum4(acc);
    __shared__ unsigned int ticket;
    if (threadIdx.x == 0) {
        double *row = scratch + kRows + 4 * (j - 1);
        for (int q = 0; q < 4; q++) row[q] = acc[q];
        __threadfence();
        ticket = atomicAdd(reinterpret_cast<unsigned int *>(scratch), 1u);
    }
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int jj = threadIdx.x; jj < n1; jj += kThreads)
        for (int q = 0; q < 4; q++) tot[q] += __ldcg(scratch + kRows + 4 * jj + q);
    block_sum4(tot);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; q++) scratch[1 + q] = sqrt(tot[q]);
        *reinterpret_cast<unsigned int *>(scratch) = 0u;
    }
}

// Device address of the scratch array on the current device.  It is looked
// up on every call: the lookup is cheap, and a cached address would go stale
// if the caller reset the device (cudaDeviceReset) and the module were
// loaded again.  The first lookup on a device loads this module there, which
// is when the array is reserved.
int scratch_address(double **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, blp_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BLP_ERR_CUDA;
    }
    *out = static_cast<double *>(p);
    return BLP_OK;
}

// True for managed memory and for device memory of the current device.  A
// device pointer of another GPU is refused: the kernel runs on the current
// device and would read memory it cannot reach.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" int blp_residual_noalloc(int N, const double *x, const double *y, double eps, const double *c1,
                                    const double *c2, const double *r, const double *f, const double *u,
                                    double *res, double *norms, void *stream) {
    if (N < 8 || N % 2 != 0 || N > BLP_NOALLOC_MAX_N) return BLP_ERR_ARG;
    if (!(eps > 0.0 && eps <= 1.0)) return BLP_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BLP_ERR_CUDA;
    const void *in[] = {x, y, c1, c2, r, f, u};
    for (const void *p : in)
        if (!p || !on_device(p, dev)) return BLP_ERR_ARG;
    if (res && !on_device(res, dev)) return BLP_ERR_ARG;
    double *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != BLP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(scratch, 0, sizeof(double), s) != cudaSuccess) return BLP_ERR_CUDA;
    k_residual_noalloc<<<N - 1, kThreads, 0, s>>>(N, x, y, eps, c1, c2, r, f, u, res, scratch);
    if (cudaGetLastError() != cudaSuccess) return BLP_ERR_CUDA;
    if (norms && cudaMemcpyAsync(norms, scratch + 1, 4 * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess)
        return BLP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BLP_ERR_CUDA;
    return BLP_OK;
}
