// blp_precond.cu -- the boundary-layer preconditioner of Sec. 3.1,
// eq. (2D blocks), applied to the row-normalised system, and its transpose.
//
//   interior block I : M_II, downstream Gauss-Seidel    -> wavefront kernel
//   edge blocks Y, X : M_YY / M_XX, ordered line solves -> line-chain kernel
//   corner block C   : M_CC, multigrid iteration (Sec. 3.2) -> wavefront
//                      smoother + fused restriction / prolongation kernels
#include "blp_common.cuh"
#include <algorithm>
#include <cstring>

#define FULL 0xffffffffu

// ---------------------------------------------------------------------------
// Wavefront kernel: downstream triangular solve on a SKEW block
//     z(a,b) = beta(a,b) - cV(a,b) zV - cH(a,b) zH
// forward (REV = false): zH = z(a+1,b) (east), zV = z(a,b+1) (north), the
//   sweep starts at the top-right node (Sec. 3.1 M_II; Sec. 3.2 smoother);
// reversed (REV = true): zH = z(a-1,b), zV = z(a,b-1), starting bottom-left
//   (the transposed sweeps of the adjoint).
// A Gauss-Seidel sweep of the full 5-point operator is this solve with
// beta = b - (couplings to the neighbours that come later in the sweep) *
// e_old, which k_gs_rhs forms in parallel beforehand; the result equals the
// sequential sweep exactly because those neighbours still hold old values.
//
// One CTA.  Warp w owns strips in processing order w, w+W, ...; lane l owns
// column 32s+l and handles diagonal d at step t (d = t forward, D-1-t
// reversed), so each step reads 32 consecutive words of beta and of the
// packed (cH, cV) pairs.  Those reads are issued RP steps ahead with
// per-lane cp.async into a shared-memory window, keeping memory latency off
// the recurrence; the step's critical path is one shuffle and one FMA.  The
// lane next to the previous strip ("head") takes that strip's boundary
// column from a shared-memory ring filled by the warp that processed it.
// All waits are bounded (BLP_ERR_TIMEOUT, no hang).
// ---------------------------------------------------------------------------
template <typename T> using Vec2T = Pair2<T>;

#define DTS_RING 128

template <typename T>
struct DtsArgs {
    Region R;
    const T *beta;
    const typename Vec2T<T>::type *pair;   // (cH, cV)
    T *out;
    const T *bnd;      // reversed interior sweep: global vector with the X/Y values west/south of the block
    Layout lay;
    const int *skip;   // nonzero -> return at once (converged)
    int *err;
};

__device__ __forceinline__ bool spin_wait_ge(volatile int *ctr, int target, volatile int *abort_flag, int *err) {
    long long n = 0;
    while (*ctr < target) {
        if (*abort_flag) return false;
        if (++n > BLP_SPIN_LIMIT) {
            *abort_flag = 1;
            atomicExch(err, BLP_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// --- bulk copies and mbarriers (inline PTX) --------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned, size a multiple of 16), completion on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// bounded wait on an mbarrier phase (BLP_ERR_TIMEOUT instead of a hang)
__device__ __forceinline__ void mbar_wait(unsigned long long *bar, unsigned parity, volatile int *abort_flag, int *err) {
    long long n = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return;
        if (++n > (BLP_SPIN_LIMIT >> 4)) {
            *abort_flag = 1;
            atomicExch(err, BLP_ERR_TIMEOUT);
            return;
        }
    }
}

// Shared-memory carve-up: per warp 2 stages of CH diagonals of beta (T) and
// (cH, cV) pairs (T2), then the inter-warp ring, counters and mbarriers.
template <typename T, int CH>
struct DtsSmem {
    typedef typename Vec2T<T>::type T2;
    static constexpr size_t stage_pairs = (size_t)CH * 32 * sizeof(T2);
    static constexpr size_t stage_beta = (size_t)CH * 32 * sizeof(T);
    static constexpr size_t per_warp = 2 * (stage_pairs + stage_beta);
    static size_t bytes(int W) {
        return (size_t)W * per_warp + (size_t)W * DTS_RING * sizeof(T) + 16 * (size_t)W + 16 * (size_t)(W + 1) + 64;
    }
};

template <typename T, bool REV, int CH, bool BND>
__global__ void __launch_bounds__(1024) k_dts(DtsArgs<T> A) {
    typedef typename Vec2T<T>::type T2;
    typedef DtsSmem<T, CH> SM;
    if (A.skip && *A.skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *mine = smem_raw + (size_t)w * SM::per_warp;
    T2 *const sp0 = reinterpret_cast<T2 *>(mine);
    T2 *const sp1 = reinterpret_cast<T2 *>(mine + SM::stage_pairs);
    T *const sb0 = reinterpret_cast<T *>(mine + 2 * SM::stage_pairs);
    T *const sb1 = reinterpret_cast<T *>(mine + 2 * SM::stage_pairs + SM::stage_beta);
    unsigned char *tailp = smem_raw + (size_t)W * SM::per_warp;
    T *ring = reinterpret_cast<T *>(tailp);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(tailp + (size_t)W * DTS_RING * sizeof(T));
    volatile int *prod = reinterpret_cast<volatile int *>(bars + 2 * W);
    volatile int *cons = prod + W;
    volatile int *abort_flag = cons + W;
    unsigned long long *const bar0 = bars + 2 * w, *const bar1 = bars + 2 * w + 1;
    if (threadIdx.x < W) { prod[threadIdx.x] = 0; cons[threadIdx.x] = 0; }
    if (threadIdx.x == 0) *abort_flag = 0;
    if (lane == 0) { mbar_init(bar0, 1); mbar_init(bar1, 1); }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();

    const Region R = A.R;
    const int S = R.S, D = R.D, my = R.my;
    const int qoff = REV ? D - (my + 31) : 0;   // padding diagonals come first in reversed order
    const int head = REV ? 0 : 31, tail = REV ? 31 : 0;
    const int waves = (S + W - 1) / W;
    const int nch = D / CH;
    const unsigned chunk_bytes = (unsigned)(SM::stage_pairs + SM::stage_beta);
    const int wn = w + 1 < W ? w + 1 : 0;
    T *const ring_in = ring + (size_t)w * DTS_RING;
    T *const ring_out = ring + (size_t)wn * DTS_RING;
    volatile int *const prod_in = prod + w;
    volatile int *const cons_in = cons + w;
    volatile int *const prod_out = prod + wn;
    volatile int *const cons_out = cons + wn;
    int in_seq = 0, out_seq = 0;
    unsigned ph0 = 0u, ph1 = 0u;

    // Strips are processed in waves of W (one per warp).  Inside a wave the
    // boundary column passes from warp w to warp w+1 through the shared
    // ring, a chunk of CH rows at a time; the first warp of a later wave
    // reads the last strip of the previous wave from global memory (complete
    // by then: the waves are separated by __syncthreads).  All waits are
    // taken by the whole warp (uniform control flow keeps the step loop
    // free of divergence).
    for (int k = 0; k < waves; k++) {
        const int sidx = w + k * W;
        if (sidx >= S) { __syncthreads(); continue; }
        const int s = REV ? sidx : S - 1 - sidx;
        const bool has_in = w > 0;
        const bool from_global = w == 0 && sidx > 0;
        const bool has_out = (w + 1 < W) && (sidx + 1 < S);
        const int sprev = REV ? s - 1 : s + 1;
        const long long sbase = R.off + (((long long)s * D) << 5);
        const T2 *const gpair = A.pair + sbase;
        const T *const gbeta = A.beta + sbase;
        if (lane == 0) {
            for (int c = 0; c < 2 && c < nch; c++) {
                const int d0 = REV ? D - (c + 1) * CH : c * CH;
                unsigned long long *bb = c ? bar1 : bar0;
                fence_proxy_async();
                mbar_arrive_expect_tx(bb, chunk_bytes);
                bulk_g2s(c ? sp1 : sp0, gpair + ((long long)d0 << 5), (unsigned)SM::stage_pairs, bb);
                bulk_g2s(c ? sb1 : sb0, gbeta + ((long long)d0 << 5), (unsigned)SM::stage_beta, bb);
            }
        }
        __syncwarp();
        T zprev = T(0);
        T *const outp = A.out + sbase + lane;
        for (int c = 0; c < nch; c++) {
            const bool st = c & 1;
            const int t0 = c * CH;
            // boundary inputs of this chunk (meaningful on the head lane), in registers
            T hz[CH];
#pragma unroll
            for (int q = 0; q < CH; q++) hz[q] = T(0);
            if (from_global) {
#pragma unroll
                for (int q = 0; q < CH; q++) {
                    const int t = t0 + q;
                    const int ktop = REV ? D - 1 - t - 31 : t;
                    const int dprev = REV ? ktop : ktop + 31;
                    if (lane == head && ktop >= 0 && ktop < my)
                        hz[q] = A.out[R.off + (((long long)sprev * D + dprev) << 5) + (REV ? 31 : 0)];
                }
            }
            mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, abort_flag, A.err);
            if (st) ph1 ^= 1u; else ph0 ^= 1u;
            if (has_in) {
                const int need = min(max(t0 + CH - qoff, 0), my);
                if (need > 0) spin_wait_ge(prod_in, in_seq + need, abort_flag, A.err);
                __threadfence_block();
#pragma unroll
                for (int q = 0; q < CH; q++) {
                    const int row = t0 + q - qoff;
                    const T v = ring_in[(in_seq + (row < 0 ? 0 : row)) & (DTS_RING - 1)];
                    hz[q] = (row >= 0 && row < my) ? v : T(0);
                }
            }
            const T2 *const pp = st ? sp1 : sp0;
            const T *const pb = st ? sb1 : sb0;
            const bool is_head = lane == head;
            T *const op = outp + ((long long)(REV ? D - 1 - t0 : t0) << 5);
            T tz[CH];
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int qi = REV ? CH - 1 - q : q;
                const T2 cpair = pp[qi * 32 + lane];
                const T beta = pb[qi * 32 + lane];
                T zH = REV ? __shfl_up_sync(FULL, zprev, 1) : __shfl_down_sync(FULL, zprev, 1);
                zH = is_head ? hz[q] : zH;
                T zV = zprev;
                if (BND) {   // reversed interior sweep: west / south neighbours in the X / Y blocks
                    const int ktop = (REV ? D - 1 - (t0 + q) : t0 + q) - 31 + lane;
                    const int a = s * 32 + lane, b = my - 1 - ktop;
                    if (ktop >= 0 && ktop < my && a < R.mx) {
                        if (a == 0) zH = A.bnd[A.lay.addr(R.i0 - 1, R.j0 + b)];
                        if (b == 0) zV = A.bnd[A.lay.addr(R.i0 + a, R.j0 - 1)];
                    }
                }
                T z = beta - cpair.y * zV;
                z = z - cpair.x * zH;
                op[REV ? -(q << 5) : (q << 5)] = z;
                tz[q] = z;
                zprev = z;
            }
            if (has_out) {
                const int last = min(t0 + CH - 31 - qoff, my);
                if (last > 0) spin_wait_ge(cons_out, out_seq + last - DTS_RING, abort_flag, A.err);
#pragma unroll
                for (int q = 0; q < CH; q++) {
                    const int row = t0 + q - 31 - qoff;
                    if (lane == tail && row >= 0 && row < my) ring_out[(out_seq + row) & (DTS_RING - 1)] = tz[q];
                }
                __threadfence_block();
                if (lane == tail) *prod_out = out_seq + min(max(t0 + CH - 31 - qoff, 0), my);
            }
            if (has_in) {
                __threadfence_block();
                if (lane == head) *cons_in = in_seq + min(max(t0 + CH - qoff, 0), my);
            }
            __syncwarp();
            if (lane == 0 && c + 2 < nch) {
                const int d0 = REV ? D - (c + 3) * CH : (c + 2) * CH;
                unsigned long long *bb = st ? bar1 : bar0;
                fence_proxy_async();
                mbar_arrive_expect_tx(bb, chunk_bytes);
                bulk_g2s(st ? sp1 : sp0, gpair + ((long long)d0 << 5), (unsigned)SM::stage_pairs, bb);
                bulk_g2s(st ? sb1 : sb0, gbeta + ((long long)d0 << 5), (unsigned)SM::stage_beta, bb);
            }
            __syncwarp();
        }
        if (has_in) in_seq += my;
        if (has_out) out_seq += my;
        __syncthreads();
    }
}

template <typename T, bool REV, int CH>
static int launch_dts_ch(blp_handle *h, const DtsArgs<T> &a, int W, int cls) {
    size_t smem = DtsSmem<T, CH>::bytes(W);
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_dts<T, REV, CH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024) != cudaSuccess ||
            cudaFuncSetAttribute(k_dts<T, REV, CH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return BLP_ERR_CUDA;
        }
        attr_set = true;
    }
    // algorithmic words per node: beta, two couplings, out
    ProfScope ps(h, cls, (double)a.R.mx * a.R.my * sizeof(T) * 4);
    if (a.bnd) k_dts<T, REV, CH, true><<<1, W * 32, smem, h->stream>>>(a);
    else k_dts<T, REV, CH, false><<<1, W * 32, smem, h->stream>>>(a);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

// Chunk length CH: 8 diagonals keeps the inter-warp hand-off lag short; a
// smaller chunk where the per-warp double buffers would not fit.
template <typename T, bool REV>
static int launch_dts(blp_handle *h, const DtsArgs<T> &a, int cls) {
    const int W = std::min(a.R.S, 32);
    const size_t cap = 225 * 1024;
    if (DtsSmem<T, 8>::bytes(W) <= cap) return launch_dts_ch<T, REV, 8>(h, a, W, cls);
    if (DtsSmem<T, 4>::bytes(W) <= cap) return launch_dts_ch<T, REV, 4>(h, a, W, cls);
    if (DtsSmem<T, 2>::bytes(W) <= cap) return launch_dts_ch<T, REV, 2>(h, a, W, cls);
    return BLP_ERR_ARG;
}

// Right-hand side of one Gauss-Seidel sweep in the wavefront form:
//   forward  beta = b - wW e_old(a-1,b) - wS e_old(a,b-1)
//   reversed beta = b - wWT e_old(a+1,b) - wST e_old(a,b+1)
template <typename T, bool REV>
__global__ void k_gs_rhs(Region R, const T *__restrict__ b, const T *__restrict__ e, const T *__restrict__ oH,
                         const T *__restrict__ oV, T *__restrict__ beta, const int *skip) {
    if (skip && *skip) return;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < R.size; q += (long long)gridDim.x * blockDim.x) {
        int a, bb;
        if (!R.coords(q, a, bb)) { beta[q] = T(0); continue; }
        T s = b[q];
        const int ah = REV ? a + 1 : a - 1, bv = REV ? bb + 1 : bb - 1;
        if (ah >= 0 && ah < R.mx) s -= oH[q] * e[R.addr(ah, bb)];
        if (bv >= 0 && bv < R.my) s -= oV[q] * e[R.addr(a, bv)];
        beta[q] = s;
    }
}

// ---------------------------------------------------------------------------
// Block-wide scan of an affine recurrence x_e = alpha_e + mu_e x_{e-1}
// (BACK = false, e ascending) or x_e = alpha_e + mu_e x_{e+1} (BACK = true),
// x = 0 outside the sequence.  Thread t owns elements [t*KPT, t*KPT+KPT).
// Warp-level Kogge-Stone over the per-thread compositions, then the warp
// totals are composed serially (few warps) through shared memory.
// ---------------------------------------------------------------------------
template <typename T, int KPT, bool BACK>
__device__ __forceinline__ void block_affine_scan(const T (&al)[KPT], const T (&mu)[KPT], T (&x)[KPT], T *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T A = T(0), M = T(1);
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        A = al[e] + mu[e] * A;
        M = mu[e] * M;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T Ap = BACK ? __shfl_down_sync(FULL, A, off) : __shfl_up_sync(FULL, A, off);
        const T Mp = BACK ? __shfl_down_sync(FULL, M, off) : __shfl_up_sync(FULL, M, off);
        const bool ok = BACK ? (lane + off < 32) : (lane >= off);
        if (ok) { A = A + M * Ap; M = M * Mp; }
    }
    const int last = BACK ? 0 : 31;
    if (lane == last) { sh[wid] = A; sh[32 + wid] = M; }
    __syncthreads();
    // carry into this warp: composition of the warps before it in sequence order
    T carry = T(0);
    if (BACK) {
        for (int v = nw - 1; v > wid; v--) carry = sh[v] + sh[32 + v] * carry;
    } else {
        for (int v = 0; v < wid; v++) carry = sh[v] + sh[32 + v] * carry;
    }
    const T Aprev = BACK ? __shfl_down_sync(FULL, A, 1) : __shfl_up_sync(FULL, A, 1);
    const T Mprev = BACK ? __shfl_down_sync(FULL, M, 1) : __shfl_up_sync(FULL, M, 1);
    const bool first = BACK ? (lane == 31) : (lane == 0);
    T xin = first ? carry : Aprev + Mprev * carry;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        xin = al[e] + mu[e] * xin;
        x[e] = xin;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Line chains (Sec. 3.1): block 0 = Y block (lines of constant x, solved
// right to left, keeping the E coupling to the line solved before and, on
// the top node, the N coupling into I), block 1 = X block (lines of constant
// y, top down, keeping the N coupling and, on the right node, the E coupling
// into I).  TRANS: the transposed block solves (Y left to right, X bottom up)
// with the couplings from the line before or, for the first line, from C.
// Both blocks run in one launch.  Each line: Thomas with the stored factors,
// both sweeps as block-wide affine scans.  The next line's data (right-hand
// side, coupling, factors, boundary value) is loaded while the current line
// is solved, so only the scans stay on the chain's critical path.
// ---------------------------------------------------------------------------
template <typename T>
struct ChainArgs {
    Layout lay;
    const T *v;
    T *z;
    const T *wE, *wN, *wET, *wNT;
    const T *lf, *lg, *lh;
    const int *skip;
};

template <typename T, int KPT>
struct LineData {
    T v[KPT], c[KPT], f[KPT], g[KPT], h[KPT], prev[KPT];
    T bval;   // boundary value (I neighbour of the last node; forward only)
};

template <typename T, int KPT, bool TRANS>
__device__ __forceinline__ void load_line(const ChainArgs<T> &A, bool isY, int nlines, int li, int e0,
                                          LineData<T, KPT> &D) {
    const Layout &lay = A.lay;
    const int L = lay.L;
    const Region &C = lay.R[0], &I = lay.R[3];
    const Region &B = isY ? lay.R[2] : lay.R[1];
    const int line = TRANS ? li : nlines - 1 - li;
    const long long base = B.off + (long long)line * L;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = e0 + q;
        if (e < L) {
            const long long s = base + e;
            D.v[q] = A.v[s];
            D.c[q] = TRANS ? (isY ? A.wET[s] : A.wNT[s]) : (isY ? A.wE[s] : A.wN[s]);
            D.f[q] = A.lf[s];
            D.g[q] = A.lg[s];
            D.h[q] = A.lh[s];
            D.prev[q] = (TRANS && li == 0) ? A.z[isY ? C.addr(L - 1, e) : C.addr(e, L - 1)] : T(0);
        } else {
            D.v[q] = T(0); D.c[q] = T(0); D.f[q] = T(1); D.g[q] = T(0); D.h[q] = T(1); D.prev[q] = T(0);
        }
    }
    D.bval = T(0);
    if (!TRANS && e0 <= L - 1 && L - 1 < e0 + KPT) {
        const long long s = base + (L - 1);
        const long long pi = isY ? I.addr(line, 0) : I.addr(0, line);
        D.bval = (isY ? A.wN[s] : A.wE[s]) * A.z[pi];
    }
}

template <typename T, int KPT, bool TRANS>
__global__ void __launch_bounds__(512) k_line_chain(ChainArgs<T> A) {
    if (A.skip && *A.skip) return;
    __shared__ T sh[64];
    const bool isY = blockIdx.x == 0;
    const Layout &lay = A.lay;
    const int L = lay.L;
    const Region &B = isY ? lay.R[2] : lay.R[1];
    const int nlines = isY ? lay.R[2].mx : lay.R[1].my;
    const int e0 = threadIdx.x * KPT;
    T zp[KPT], al[KPT], mu[KPT], y[KPT];
#pragma unroll
    for (int q = 0; q < KPT; q++) zp[q] = T(0);
    LineData<T, KPT> cur, nxt;
    if (nlines > 0) load_line<T, KPT, TRANS>(A, isY, nlines, 0, e0, cur);
    for (int li = 0; li < nlines; li++) {
        if (li + 1 < nlines) load_line<T, KPT, TRANS>(A, isY, nlines, li + 1, e0, nxt);
        const int line = TRANS ? li : nlines - 1 - li;
        const long long base = B.off + (long long)line * L;
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const T prev = (TRANS && li == 0) ? cur.prev[q] : zp[q];
            T d = cur.v[q] - cur.c[q] * prev;
            if (!TRANS && e0 + q == L - 1) d -= cur.bval;
            al[q] = d;
            mu[q] = cur.f[q];
        }
        block_affine_scan<T, KPT, false>(al, mu, y, sh);
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            al[q] = cur.g[q] * y[q];
            mu[q] = cur.h[q];
        }
        block_affine_scan<T, KPT, true>(al, mu, zp, sh);
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int e = e0 + q;
            if (e < L) A.z[base + e] = zp[q];
            else zp[q] = T(0);
        }
        cur = nxt;
    }
}

template <typename T, bool TRANS>
static int launch_chains(blp_handle *h, const Coefs<T> &c, const T *v, T *z, const int *skip) {
    ChainArgs<T> a;
    a.lay = h->lay; a.v = v; a.z = z;
    a.wE = c.wE; a.wN = c.wN; a.wET = c.wET; a.wNT = c.wNT;
    a.lf = TRANS ? c.lfT : c.lf; a.lg = TRANS ? c.lgT : c.lg; a.lh = TRANS ? c.lhT : c.lh;
    a.skip = skip;
    int L = h->L;
    // per line node: v, coupling, three factors, z = 6 words
    ProfScope ps(h, KC_LINE_CHAIN, (double)(h->lay.R[1].size + h->lay.R[2].size) * sizeof(T) * 6);
    if (L <= 2048) {
        int nt = ((L + 3) / 4 + 31) / 32 * 32;
        k_line_chain<T, 4, TRANS><<<2, nt, 0, h->stream>>>(a);
    } else {
        int nt = ((L + 15) / 16 + 31) / 32 * 32;
        k_line_chain<T, 16, TRANS><<<2, nt, 0, h->stream>>>(a);
    }
    LAUNCH_CHECK(h);
    return BLP_OK;
}

// ---------------------------------------------------------------------------
// Corner right-hand side (Sec. 3.1 block back substitution):
//   b_C = v_C - A_CX z_X - A_CY z_Y (normalised): only the top row of C
//   couples to X (N) and the right column to Y (E).  The level-0 block has
//   the same SKEW geometry as the C block of the global vectors (both start
//   at slot 0), so slots coincide.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_corner_rhs(Layout lay, const T *__restrict__ v, const T *__restrict__ z, const T *__restrict__ wE,
                             const T *__restrict__ wN, T *__restrict__ b0, const int *skip) {
    if (skip && *skip) return;
    const Region &C = lay.R[0];
    const int L = lay.L;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.size; q += (long long)gridDim.x * blockDim.x) {
        int a, b;
        if (!C.coords(q, a, b)) { b0[q] = T(0); continue; }
        T s = v[q];
        if (b == L - 1) s -= wN[q] * z[lay.R[1].addr(a, 0)];
        if (a == L - 1) s -= wE[q] * z[lay.R[2].addr(0, b)];
        b0[q] = s;
    }
}

// ---------------------------------------------------------------------------
// Corner multigrid kernels (Sec. 3.2, two exponential layers): full
// coarsening, bilinear P, restriction P^T in finite-element scaling.
// For the row-normalised operator the scaling weight is omega = hb*kb*aC:
//   forward   b_c = omega_c^-1 P^T (omega_f r_f),  e_f += P e_c
//   transpose b_c = P^T r_f,                       e_f += omega_f P (omega_c^-1 e_c)
// (the exact transpose of the forward cycle).
// ---------------------------------------------------------------------------
template <typename T, bool TRANS>
__device__ __forceinline__ T level_residual(const Level<T> &Lv, const T *__restrict__ b, const T *__restrict__ e,
                                            int a, int bb) {
    const Region &R = Lv.R;
    const long long p = R.addr(a, bb);
    T s = e[p];
    if (!TRANS) {
        if (a > 0) s += Lv.wW[p] * e[R.addr(a - 1, bb)];
        if (a < R.mx - 1) s += Lv.wE[p] * e[R.addr(a + 1, bb)];
        if (bb > 0) s += Lv.wS[p] * e[R.addr(a, bb - 1)];
        if (bb < R.my - 1) s += Lv.wN[p] * e[R.addr(a, bb + 1)];
    } else {
        if (a > 0) s += Lv.wET[p] * e[R.addr(a - 1, bb)];
        if (a < R.mx - 1) s += Lv.wWT[p] * e[R.addr(a + 1, bb)];
        if (bb > 0) s += Lv.wNT[p] * e[R.addr(a, bb - 1)];
        if (bb < R.my - 1) s += Lv.wST[p] * e[R.addr(a, bb + 1)];
    }
    return b[p] - s;
}

template <typename T, bool TRANS>
__global__ void k_mg_restrict(Level<T> F, const T *__restrict__ bf, const T *__restrict__ ef, Level<T> Cc,
                              T *__restrict__ bc, T *__restrict__ ec, const int *skip) {
    if (skip && *skip) return;
    const Region &RC = Cc.R, &RF = F.R;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < RC.size; q += (long long)gridDim.x * blockDim.x) {
        ec[q] = T(0);
        int A, B;
        if (!RC.coords(q, A, B)) { bc[q] = T(0); continue; }
        const int a0 = 2 * A + 1, b0 = 2 * B + 1;
        T sum = T(0);
#pragma unroll
        for (int db = -1; db <= 1; db++) {
            const int bb = b0 + db;
            if (bb < 0 || bb >= RF.my) continue;
            const T wy = db == 0 ? T(1) : T(0.5);
#pragma unroll
            for (int da = -1; da <= 1; da++) {
                const int a = a0 + da;
                if (a < 0 || a >= RF.mx) continue;
                const T wx = da == 0 ? T(1) : T(0.5);
                T r = level_residual<T, TRANS>(F, bf, ef, a, bb);
                if (!TRANS) r *= F.omega[RF.addr(a, bb)];
                sum += wx * wy * r;
            }
        }
        bc[q] = TRANS ? sum : sum / Cc.omega[q];
    }
}

template <typename T, bool TRANS>
__global__ void k_mg_prolong(Level<T> F, T *__restrict__ ef, Level<T> Cc, const T *__restrict__ ec, const int *skip) {
    if (skip && *skip) return;
    const Region &RF = F.R, &RC = Cc.R;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < RF.size; q += (long long)gridDim.x * blockDim.x) {
        int a, b;
        if (!RF.coords(q, a, b)) continue;
        const int I = a + 1, J = b + 1;   // 1-based fine node
        auto cval = [&](int Ic, int Jc) -> T {
            if (Ic < 1 || Jc < 1 || Ic > RC.mx || Jc > RC.my) return T(0);
            const long long pc = RC.addr(Ic - 1, Jc - 1);
            return TRANS ? ec[pc] / Cc.omega[pc] : ec[pc];
        };
        T v;
        const bool Ie = !(I & 1), Je = !(J & 1);
        if (Ie && Je) v = cval(I / 2, J / 2);
        else if (!Ie && Je) v = T(0.5) * (cval((I - 1) / 2, J / 2) + cval((I + 1) / 2, J / 2));
        else if (Ie && !Je) v = T(0.5) * (cval(I / 2, (J - 1) / 2) + cval(I / 2, (J + 1) / 2));
        else v = T(0.25) * (cval((I - 1) / 2, (J - 1) / 2) + cval((I + 1) / 2, (J - 1) / 2) +
                            cval((I - 1) / 2, (J + 1) / 2) + cval((I + 1) / 2, (J + 1) / 2));
        if (TRANS) v *= F.omega[q];
        ef[q] += v;
    }
}

// Squared norm of the stopping residual of the corner iteration (FE
// scaling): forward ||omega (b - A e)||, transpose ||hb kb (b - A^T e)||.
// mode 0: of b alone (initial value), mode 1: of the residual.
// Partial sums per block (FP64) -> k_corner_finish.
template <typename T, bool TRANS>
__global__ void k_corner_norm(Level<T> Lv, const T *__restrict__ b, const T *__restrict__ e, int mode,
                              double *partials, const int *skip) {
    if (skip && *skip) return;
    const Region &R = Lv.R;
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < R.size; q += (long long)gridDim.x * blockDim.x) {
        int a, bb;
        if (!R.coords(q, a, bb)) continue;
        T r = mode == 0 ? b[q] : level_residual<T, TRANS>(Lv, b, e, a, bb);
        double wr = (double)(TRANS ? Lv.dfe[q] : Lv.omega[q]) * (double)r;
        acc += wr * wr;
    }
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

// mode 0: red[0] = ||b||^2 / reduction^2, flags[0] = (||b|| == 0), flags[1] = 0
// mode 1: flags[1]++, flags[0] = (||r||^2 <= red[0]) or cycles reached the cap
__global__ void k_corner_finish(double *partials, int nb, DevState *st, int mode, double red2, int maxc) {
    if (st->flags[0] && mode == 1) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += partials[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(FULL, s, off);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            st->red[0] = s / red2;
            st->flags[0] = (s == 0.0);
            st->flags[1] = 0;
        } else {
            st->flags[1] += 1;
            if (s <= st->red[0] || st->flags[1] >= maxc) st->flags[0] = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Fused coarse levels (Sec. 3.2 cycle below a size where a level fits in
// shared memory).  One CTA runs the V(1,1) cycle from level l0 to the
// coarsest and back: every level's iterate and right-hand side live in
// shared memory (natural row-major layout), Gauss-Seidel is an in-place
// anti-diagonal wavefront (the sequential downstream order exactly: a node
// reads its E/N neighbours from the diagonal just updated and its W/S
// neighbours still old), restriction and prolongation are CTA-parallel.
// full = 1: l0 = 0 and the whole stationary iteration of M_CC (cycles and
// the FE-scaled stopping test) runs here; full = 0: one cycle from a zero
// iterate for the coarse-grid correction of level l0 - 1.
// ---------------------------------------------------------------------------
template <typename T>
struct CoarseArgs {
    int l0, nlev;                     // levels l0 .. nlev-1 are handled here
    int m[BLP_MAXLEV];
    const T *nat[BLP_MAXLEV];         // 10 natural arrays per level (see Level::nat)
    const T *b_in;                    // right-hand side of level l0 (its SKEW layout)
    T *e_out;                         // result on level l0 (SKEW layout)
    Region R0;                        // level l0 SKEW region
    int full, fixed_cycles, max_cycles;
    double red2;                      // reduction factor squared
    DevState *st;
    const int *skip;
};

// Shared-memory image of one level inside the fused kernel (natural layout):
// e, b, the four couplings of the sweep direction (forward wW, wE, wS, wN;
// transpose wET, wWT, wNT, wST), omega = hb*kb*aC (restriction of the
// forward cycle, prolongation of the transposed one) and the weight of the
// stopping norm (forward omega, transpose hb*kb).
template <typename T>
struct CLev {
    int m;
    T *e, *b, *cw, *ce, *cs, *cn, *om, *wt;
};

// r = b - Op e at node (a, b) of a level (Op: normalised operator, or its transpose)
template <typename T>
__device__ __forceinline__ T coarse_residual(const CLev<T> L, int a, int bb) {
    const int m = L.m, k = bb * m + a;
    T s = L.e[k];
    if (a > 0) s += L.cw[k] * L.e[k - 1];
    if (a < m - 1) s += L.ce[k] * L.e[k + 1];
    if (bb > 0) s += L.cs[k] * L.e[k - m];
    if (bb < m - 1) s += L.cn[k] * L.e[k + m];
    return L.b[k] - s;
}

// One downstream Gauss-Seidel sweep of a level, as an anti-diagonal wavefront
// over shared memory; thread a owns column a (in-place: a node reads its E/N
// neighbours from the diagonal just updated and its W/S neighbours still
// old, which is the sequential order exactly).  Levels up to 32 wide run in
// one warp.
template <typename T, bool TRANS>
__device__ __forceinline__ void coarse_gs_body(const CLev<T> L, int a, bool warp_only) {
    const int m = L.m;
    for (int step = 0; step < 2 * m - 1; step++) {
        const int b = (TRANS ? step : 2 * m - 2 - step) - a;
        if (a < m && b >= 0 && b < m) {
            const int k = b * m + a;
            T s = L.b[k];
            if (a > 0) s -= L.cw[k] * L.e[k - 1];
            if (a < m - 1) s -= L.ce[k] * L.e[k + 1];
            if (b > 0) s -= L.cs[k] * L.e[k - m];
            if (b < m - 1) s -= L.cn[k] * L.e[k + m];
            L.e[k] = s;
        }
        if (warp_only) __syncwarp(); else __syncthreads();
    }
}

template <typename T, bool TRANS>
__device__ __forceinline__ void coarse_gs(const CLev<T> L) {
    if (L.m <= 32) {
        if (threadIdx.x < 32) coarse_gs_body<T, TRANS>(L, threadIdx.x, true);
        __syncthreads();
    } else {
        coarse_gs_body<T, TRANS>(L, threadIdx.x, false);   // m <= blockDim.x
    }
}

template <typename T>
__device__ __forceinline__ T coarse_val(const T *ec, int mc, int I, int J) {
    return (I < 1 || J < 1 || I > mc || J > mc) ? T(0) : ec[(J - 1) * mc + (I - 1)];
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_mg_coarse(CoarseArgs<T> A) {
    if (A.skip && *A.skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[8];
    CLev<T> LV[BLP_MAXLEV];
    {
        T *p = reinterpret_cast<T *>(smem_raw);
        for (int l = A.l0; l < A.nlev; l++) {
            const int m = A.m[l], n = m * m;
            CLev<T> &L = LV[l];
            L.m = m;
            L.e = p; p += n;
            L.b = p; p += n;
            L.cw = p; p += n; L.ce = p; p += n; L.cs = p; p += n; L.cn = p; p += n; L.om = p; p += n;
            L.wt = TRANS ? p : L.om;
            if (TRANS) p += n;
            const T *nat = A.nat[l];
            const int q0 = TRANS ? 4 : 0;
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                L.cw[k] = nat[(long long)(q0 + 0) * n + k];
                L.ce[k] = nat[(long long)(q0 + 1) * n + k];
                L.cs[k] = nat[(long long)(q0 + 2) * n + k];
                L.cn[k] = nat[(long long)(q0 + 3) * n + k];
                L.om[k] = nat[(long long)8 * n + k];
                if (TRANS) L.wt[k] = nat[(long long)9 * n + k];
            }
        }
    }
    const int l0 = A.l0, last = A.nlev - 1, m0 = A.m[l0];
    const Region R0 = A.R0;
    for (int k = threadIdx.x; k < m0 * m0; k += blockDim.x) {
        LV[l0].b[k] = A.b_in[R0.addr(k % m0, k / m0)];
        LV[l0].e[k] = T(0);
    }
    __syncthreads();

    auto vcycle = [&]() {
        for (int l = l0; l < last; l++) {
            const CLev<T> F = LV[l], Cc = LV[l + 1];
            const int m = F.m, mc = Cc.m;
            coarse_gs<T, TRANS>(F);
            // restriction of the residual: forward b_c = omega_c^-1 P^T omega_f r, transpose b_c = P^T r
            for (int q = threadIdx.x; q < mc * mc; q += blockDim.x) {
                const int a0 = 2 * (q % mc) + 1, b0 = 2 * (q / mc) + 1;
                T sum = T(0);
                for (int db = -1; db <= 1; db++) {
                    const int bb = b0 + db;
                    if (bb < 0 || bb >= m) continue;
                    for (int da = -1; da <= 1; da++) {
                        const int a = a0 + da;
                        if (a < 0 || a >= m) continue;
                        T r = coarse_residual<T>(F, a, bb);
                        if (!TRANS) r *= F.om[bb * m + a];
                        sum += (da == 0 ? T(1) : T(0.5)) * (db == 0 ? T(1) : T(0.5)) * r;
                    }
                }
                Cc.b[q] = TRANS ? sum : sum / Cc.om[q];
                Cc.e[q] = T(0);
            }
            __syncthreads();
        }
        for (int s4 = 0; s4 < 4; s4++) coarse_gs<T, TRANS>(LV[last]);
        for (int l = last - 1; l >= l0; l--) {
            const CLev<T> F = LV[l], Cc = LV[l + 1];
            const int m = F.m, mc = Cc.m;
            for (int k = threadIdx.x; k < m * m; k += blockDim.x) {
                const int I = k % m + 1, J = k / m + 1;
                auto cv = [&](int Ic, int Jc) -> T {
                    if (Ic < 1 || Jc < 1 || Ic > mc || Jc > mc) return T(0);
                    const int kc = (Jc - 1) * mc + (Ic - 1);
                    return TRANS ? Cc.e[kc] / Cc.om[kc] : Cc.e[kc];
                };
                T v;
                const bool Ie = !(I & 1), Je = !(J & 1);
                if (Ie && Je) v = cv(I / 2, J / 2);
                else if (!Ie && Je) v = T(0.5) * (cv((I - 1) / 2, J / 2) + cv((I + 1) / 2, J / 2));
                else if (Ie && !Je) v = T(0.5) * (cv(I / 2, (J - 1) / 2) + cv(I / 2, (J + 1) / 2));
                else v = T(0.25) * (cv((I - 1) / 2, (J - 1) / 2) + cv((I + 1) / 2, (J - 1) / 2) +
                                    cv((I - 1) / 2, (J + 1) / 2) + cv((I + 1) / 2, (J + 1) / 2));
                if (TRANS) v *= F.om[k];
                F.e[k] += v;
            }
            __syncthreads();
            coarse_gs<T, TRANS>(F);
        }
    };

    if (!A.full) {
        vcycle();
    } else {
        // stationary iteration of M_CC with the stopping test on the FE-scaled residual
        const CLev<T> L0 = LV[l0];
        auto norm2 = [&](int resid) -> double {
            const int n = m0 * m0;
            double acc = 0.0;
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                const T r = resid ? coarse_residual<T>(L0, k % m0, k / m0) : L0.b[k];
                const double wr = (double)L0.wt[k] * (double)r;
                acc += wr * wr;
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
            __syncthreads();
            return tot;
        };
        int cyc = 0;
        if (A.fixed_cycles > 0) {
            for (; cyc < A.fixed_cycles; cyc++) vcycle();
        } else {
            const double thresh = norm2(0) / A.red2;
            if (thresh > 0.0) {
                while (cyc < A.max_cycles) {
                    vcycle();
                    cyc++;
                    if (norm2(1) <= thresh) break;
                }
            }
        }
        if (threadIdx.x == 0 && A.st) {
            A.st->flags[1] = cyc;
            A.st->flags[0] = 1;
            atomicMax(&A.st->flags[3], cyc);
        }
    }
    for (int k = threadIdx.x; k < m0 * m0; k += blockDim.x) A.e_out[R0.addr(k % m0, k / m0)] = LV[l0].e[k];
}

template <typename T>
static size_t coarse_smem(const Hierarchy<T> &H, int l0) {
    size_t b = 0;
    for (int l = l0; l < H.nlev; l++) b += 8 * sizeof(T) * (size_t)H.lev[l].R.mx * H.lev[l].R.mx;
    return b;
}

// first level handled by the fused coarse kernel (-1: none)
template <typename T>
static int coarse_start(const Hierarchy<T> &H) {
    for (int l = 0; l < H.nlev; l++)
        if (H.lev[l].nat && coarse_smem(H, l) <= 200 * 1024) return l;
    return -1;
}

template <typename T, bool TRANS>
static int launch_coarse(blp_handle *h, Hierarchy<T> &H, int l0, const T *b_in, T *e_out, int full, const int *skip) {
    CoarseArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.l0 = l0; a.nlev = H.nlev;
    for (int l = 0; l < H.nlev; l++) { a.m[l] = H.lev[l].R.mx; a.nat[l] = H.lev[l].nat; }
    a.b_in = b_in; a.e_out = e_out; a.R0 = H.lev[l0].R;
    a.full = full; a.fixed_cycles = h->p.corner_fixed_cycles; a.max_cycles = h->p.corner_max_cycles;
    a.red2 = h->p.corner_reduction * h->p.corner_reduction;
    a.st = h->dev; a.skip = skip;
    const size_t smem = coarse_smem(H, l0);
    static bool attr = false;
    if (!attr) {
        // dynamic bytes this kernel ever asks for (coarse_start caps them at 200 KB); it also
        // has a little static shared memory, so the opt-in maximum itself would be rejected
        if (cudaFuncSetAttribute(k_mg_coarse<T, TRANS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return BLP_ERR_CUDA;
        }
        attr = true;
    }
    double bytes = 0.0;
    for (int l = l0; l < H.nlev; l++) bytes += 14.0 * sizeof(T) * H.lev[l].R.mx * H.lev[l].R.mx;
    ProfScope ps(h, KC_MG_COARSE, bytes);
    k_mg_coarse<T, TRANS><<<1, 256, smem, h->stream>>>(a);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
template <typename T> static Coefs<T> &coefs_of(blp_handle *h);
template <> Coefs<double> &coefs_of<double>(blp_handle *h) { return h->cd; }
template <> Coefs<float> &coefs_of<float>(blp_handle *h) { return h->cf; }
template <typename T> static Hierarchy<T> &hier_of(blp_handle *h);
template <> Hierarchy<double> &hier_of<double>(blp_handle *h) { return h->hd; }
template <> Hierarchy<float> &hier_of<float>(blp_handle *h) { return h->hf; }

template <typename T, bool TRANS>
struct Cycler {
    blp_handle *h;
    Hierarchy<T> *H;
    int cur[BLP_MAXLEV];
    bool zero[BLP_MAXLEV];   // current iterate of the level is known to be 0
    const T *b0;             // level-0 right-hand side
    const int *skip;
    int l0c;                 // first level of the fused coarse kernel (-1: none)

    int gs(int l, const T *b) {
        Level<T> &Lv = H->lev[l];
        const T *beta = b;
        if (!zero[l]) {
            ProfScope ps(h, KC_GS_RHS, (double)Lv.R.mx * Lv.R.my * sizeof(T) * 5);   // b, e, 2 couplings, beta
            k_gs_rhs<T, TRANS><<<grid_for(Lv.R.size, 256), 256, 0, h->stream>>>(
                Lv.R, b, Lv.e[cur[l]], TRANS ? Lv.wWT : Lv.wW, TRANS ? Lv.wST : Lv.wS, Lv.beta, skip);
            LAUNCH_CHECK(h);
            beta = Lv.beta;
        }
        DtsArgs<T> a;
        a.R = Lv.R; a.beta = beta; a.pair = TRANS ? Lv.pR : Lv.pF; a.out = Lv.e[cur[l] ^ 1];
        a.bnd = nullptr; a.lay = h->lay; a.skip = skip; a.err = h->err;
        int rc = launch_dts<T, TRANS>(h, a, KC_DTS_GS);
        cur[l] ^= 1;
        zero[l] = false;
        return rc;
    }
    int vcycle(int l) {
        Level<T> &Lv = H->lev[l];
        const T *b = l == 0 ? b0 : Lv.b;
        if (l == l0c && l > 0) {   // coarse-grid correction from a zero iterate, fused
            int rc = launch_coarse<T, TRANS>(h, *H, l, b, Lv.e[cur[l]], 0, skip);
            zero[l] = false;
            return rc;
        }
        if (l == H->nlev - 1) {
            for (int s = 0; s < 4; s++) { int rc = gs(l, b); if (rc) return rc; }
            return BLP_OK;
        }
        int rc = gs(l, b);
        if (rc) return rc;
        Level<T> &Cn = H->lev[l + 1];
        {
            // fine b, e, 4 couplings, omega once each; coarse b written
            ProfScope ps(h, KC_MG_RESTRICT, ((double)Lv.R.mx * Lv.R.my * 7 + (double)Cn.R.mx * Cn.R.my * 2) * sizeof(T));
            k_mg_restrict<T, TRANS><<<grid_for(Cn.R.size, 256), 256, 0, h->stream>>>(Lv, b, Lv.e[cur[l]], Cn, Cn.b,
                                                                                    Cn.e[cur[l + 1]], skip);
            LAUNCH_CHECK(h);
        }
        zero[l + 1] = true;
        rc = vcycle(l + 1);
        if (rc) return rc;
        {
            // fine e read + written, coarse e (and omega) read
            ProfScope ps(h, KC_MG_PROLONG, ((double)Lv.R.mx * Lv.R.my * (TRANS ? 3 : 2) + (double)Cn.R.mx * Cn.R.my * (TRANS ? 2 : 1)) * sizeof(T));
            k_mg_prolong<T, TRANS><<<grid_for(Lv.R.size, 256), 256, 0, h->stream>>>(Lv, Lv.e[cur[l]], Cn, Cn.e[cur[l + 1]], skip);
            LAUNCH_CHECK(h);
        }
        return gs(l, b);
    }
};

// M_CC^{-1} b0 (or M_CC^{-T} b0) by the stationary multigrid iteration from
// e = 0; the result is left in the returned level-0 buffer.
template <typename T, bool TRANS>
static int corner_solve(blp_handle *h, const T *b0, T **result, int *cycles_out) {
    Hierarchy<T> &H = hier_of<T>(h);
    const int l0c = coarse_start(H);
    if (l0c == 0) {
        // the whole corner iteration fits one CTA: a single launch, cycle count kept on the device
        int rc = launch_coarse<T, TRANS>(h, H, 0, b0, H.lev[0].e[0], 1, nullptr);
        *result = H.lev[0].e[0];
        if (cycles_out) *cycles_out = -1;
        return rc;
    }
    Cycler<T, TRANS> cy;
    cy.h = h; cy.H = &H; cy.b0 = b0; cy.l0c = l0c;
    for (int l = 0; l < H.nlev; l++) { cy.cur[l] = 0; cy.zero[l] = false; }
    cy.zero[0] = true;
    Level<T> &L0 = H.lev[0];
    CUDA_TRY(cudaMemsetAsync(L0.e[0], 0, sizeof(T) * L0.R.size, h->stream));
    const int fixed = h->p.corner_fixed_cycles;
    int cycles = 0;
    if (fixed > 0) {
        cy.skip = nullptr;
        for (int c = 0; c < fixed; c++) { int rc = cy.vcycle(0); if (rc) return rc; }
        cycles = fixed;
    } else {
        int *done = h->dev->flags;   // flags[0]
        const int nb = 148;
        const double red2 = h->p.corner_reduction * h->p.corner_reduction;
        cy.skip = nullptr;
        {
            ProfScope ps(h, KC_CORNER_NORM, (double)L0.R.mx * L0.R.my * 2 * sizeof(T));
            k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[0], 0, h->partials, nullptr);
            LAUNCH_CHECK(h);
            k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 0, red2, h->p.corner_max_cycles);
            LAUNCH_CHECK(h);
        }
        cy.skip = done;
        int batch = std::max(2, std::min(h->last_cycles > 0 ? h->last_cycles : 6, h->p.corner_max_cycles));
        int enq = 0;
        for (;;) {
            for (int c = 0; c < batch && enq < h->p.corner_max_cycles; c++, enq++) {
                int rc = cy.vcycle(0);
                if (rc) return rc;
                ProfScope ps(h, KC_CORNER_NORM, (double)L0.R.mx * L0.R.my * 7 * sizeof(T));
                k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[cy.cur[0]], 1, h->partials, done);
                LAUNCH_CHECK(h);
                k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 1, red2, h->p.corner_max_cycles);
                LAUNCH_CHECK(h);
            }
            CUDA_TRY(cudaMemcpyAsync(h->host_state, h->dev, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            if (h->host_state->flags[0] || enq >= h->p.corner_max_cycles) break;
            batch = 2;
        }
        cycles = h->host_state->flags[1];
        h->last_cycles = cycles + 1;
    }
    *result = L0.e[cy.cur[0]];
    if (cycles_out) *cycles_out = cycles;
    return BLP_OK;
}

// z = (D^-1 M)^-1 v, or (D^-1 M)^-T v, both in the region-major layout.
template <typename T>
int precond_apply(blp_handle *h, const T *v, T *z, int trans, int *cycles) {
    Coefs<T> &c = coefs_of<T>(h);
    Hierarchy<T> &H = hier_of<T>(h);
    const Layout &lay = h->lay;
    const Region &C = lay.R[0];
    int rc;
    if (!trans) {
        // I block: downstream Gauss-Seidel sweep of M_II (E and N kept)
        DtsArgs<T> a;
        a.R = lay.R[3]; a.beta = v; a.pair = c.pF; a.out = z;
        a.bnd = nullptr; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, false>(h, a, KC_DTS_INTERIOR))) return rc;
        // Y and X blocks
        if ((rc = launch_chains<T, false>(h, c, v, z, nullptr))) return rc;
        // C block
        T *b0 = H.lev[0].b;
        {
            ProfScope ps(h, KC_LAYOUT);
            k_corner_rhs<T><<<grid_for(C.size, 256), 256, 0, h->stream>>>(lay, v, z, c.wE, c.wN, b0, nullptr);
            LAUNCH_CHECK(h);
        }
        T *e = nullptr;
        if ((rc = corner_solve<T, false>(h, b0, &e, cycles))) return rc;
        {
            ProfScope ps(h, KC_LAYOUT);
            CUDA_TRY(cudaMemcpyAsync(z + C.off, e, sizeof(T) * C.size, cudaMemcpyDeviceToDevice, h->stream));
        }
    } else {
        T *e = nullptr;
        if ((rc = corner_solve<T, true>(h, v + C.off, &e, cycles))) return rc;
        {
            ProfScope ps(h, KC_LAYOUT);
            CUDA_TRY(cudaMemcpyAsync(z + C.off, e, sizeof(T) * C.size, cudaMemcpyDeviceToDevice, h->stream));
        }
        if ((rc = launch_chains<T, true>(h, c, v, z, nullptr))) return rc;
        DtsArgs<T> a;
        a.R = lay.R[3]; a.beta = v; a.pair = c.pR; a.out = z;
        a.bnd = z; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, true>(h, a, KC_DTS_INTERIOR))) return rc;
    }
    return BLP_OK;
}

template int precond_apply<double>(blp_handle *, const double *, double *, int, int *);
template int precond_apply<float>(blp_handle *, const float *, float *, int, int *);
