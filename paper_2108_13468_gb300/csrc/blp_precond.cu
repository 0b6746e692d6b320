// blp_precond.cu -- the boundary-layer preconditioner of Sec. 3.1,
// eq. (2D blocks), applied to the row-normalised system, and its transpose.
//
//   interior block I : M_II, downstream Gauss-Seidel    -> wavefront kernel
//   edge blocks Y, X : M_YY / M_XX, ordered line solves -> line-chain kernel
//   corner block C   : M_CC, multigrid iteration (Sec. 3.2) -> wavefront
//                      smoother + fused restriction / prolongation kernels
#include "blp_common.cuh"
#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

#define FULL 0xffffffffu

#include "blp_dts.cuh"

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
// nw: the warps taking part (all of the block's by default); with one warp
// the scan uses no block barrier, so other warps of the block may run other code.
template <typename T, int KPT, bool BACK>
__device__ __forceinline__ void block_affine_scan(const T (&al)[KPT], const T (&mu)[KPT], T (&x)[KPT], T *sh,
                                                  int nw = -1) {
    if (nw < 0) nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    if (nw > 1) {
        if (lane == last) { sh[wid] = A; sh[32 + wid] = M; }
        __syncthreads();
    }
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
    if (nw > 1) __syncthreads();
}

// The multipliers of block_affine_scan do not depend on the right-hand side:
// thread t's product M of its KPT multipliers (scan order), the M it holds
// before each of the five Kogge-Stone levels, its final M (the warp total on
// the last lane) and its neighbour's final M.  scan_multipliers computes the
// seven values with exactly the products block_affine_scan forms;
// block_affine_scan_pre then runs the A part of the same scan with them.
template <typename T, int KPT, bool BACK>
__device__ __forceinline__ void scan_multipliers(const T (&mu)[KPT], T (&pre)[7]) {
    const int lane = threadIdx.x & 31;
    T M = T(1);
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        M = mu[e] * M;
    }
    int lvl = 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        pre[lvl++] = M;
        const T Mp = BACK ? __shfl_down_sync(FULL, M, off) : __shfl_up_sync(FULL, M, off);
        const bool ok = BACK ? (lane + off < 32) : (lane >= off);
        if (ok) M = M * Mp;
    }
    pre[5] = M;
    pre[6] = BACK ? __shfl_down_sync(FULL, M, 1) : __shfl_up_sync(FULL, M, 1);
}

// sh: 64 values of shared memory, not the buffer of the scan just before
// (the warp totals of a scan stay readable until the scan after next).
template <typename T, int KPT, bool BACK>
__device__ __forceinline__ void block_affine_scan_pre(const T (&al)[KPT], const T (&mu)[KPT], const T (&pre)[7],
                                                      T (&x)[KPT], T *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T A = T(0);
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        A = al[e] + mu[e] * A;
    }
    int lvl = 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T Ap = BACK ? __shfl_down_sync(FULL, A, off) : __shfl_up_sync(FULL, A, off);
        const bool ok = BACK ? (lane + off < 32) : (lane >= off);
        if (ok) A = A + pre[lvl] * Ap;
        lvl++;
    }
    const int last = BACK ? 0 : 31;
    if (nw > 1) {
        if (lane == last) { sh[wid] = A; sh[32 + wid] = pre[5]; }
        __syncthreads();
    }
    // carry into this warp; the first warp total before it enters as is
    T carry = T(0);
    if (BACK) {
        if (wid < nw - 1) carry = sh[nw - 1];
        for (int v = nw - 2; v > wid; v--) carry = sh[v] + sh[32 + v] * carry;
    } else {
        if (wid > 0) carry = sh[0];
        for (int v = 1; v < wid; v++) carry = sh[v] + sh[32 + v] * carry;
    }
    const T Aprev = BACK ? __shfl_down_sync(FULL, A, 1) : __shfl_up_sync(FULL, A, 1);
    const bool first = BACK ? (lane == 31) : (lane == 0);
    T xin = first ? carry : Aprev + pre[6] * carry;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        xin = al[e] + mu[e] * xin;
        x[e] = xin;
    }
    // no closing barrier: callers alternate two sh buffers between
    // consecutive scans, and the next scan's barrier orders the reuse
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
    const T *pre;   // precomputed scan multipliers of this direction (k_line_chain2)
    int nlmax;      // lines per block in the pre layout
    const int *skip;
    int *err;       // k_line_chain2: BLP_ERR_TIMEOUT if a stage copy never arrives
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

// Line chains for L <= 2048 with 16-byte aligned lines (L * sizeof(T) a
// multiple of 16).  The line data (right-hand side, coupling, three factors
// and, in FP64, the scan multipliers) arrive in NS shared-memory stages, NS-1
// lines ahead of the solve.  Thread t owns the KPT consecutive nodes
// [t*KPT, t*KPT+KPT) of a line.  NW = 1 keeps both scans inside one warp (no
// CTA barrier).
// - FP64 (USEPRE): thread 0 issues one bulk copy per array (cp.async.bulk, one
//   mbarrier per stage, bounded waits) into dense arrays.  Per-thread 16-byte
//   copies cost the critical warp ~1100 cycles of issue per line (measured);
//   the dense layout costs 2-way bank conflicts on the 32-byte segments.
// - FP32: each thread copies 16-byte pieces with cp.async into arrays whose
//   KPT-element segments are each followed by 16 bytes of padding, so the
//   vector reads are conflict-free (a dense layout gives 16-element segments
//   4-way conflicts and measured 43% slower).
// The boundary term of the last node (two words) comes by cp.async to the
// thread that owns that node.
template <typename T, int KPT, int NW, bool USEPRE>
struct ChainSmem {
    static constexpr int VEC = 16 / sizeof(T);         // elements per 16 bytes
    static constexpr int LP = 32 * NW * KPT;           // line length the threads cover
    static constexpr int SEG = USEPRE ? KPT : KPT + VEC;   // stride of a thread's segment
    static constexpr int LPP = LP / KPT * SEG;         // array length in the stage
    static constexpr int PRE = USEPRE ? 14 * 32 * NW : 0;   // scan multipliers: 2 scans x 7 per thread
    static constexpr size_t stage_elems = (size_t)5 * LPP + PRE + VEC;   // arrays, multipliers, boundary term
    static constexpr size_t stage = stage_elems * sizeof(T);
    static __device__ __forceinline__ int at(int e) { return e / KPT * SEG + e % KPT; }
};

__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_word(T *dst, const T *src) {
    if constexpr (sizeof(T) == 4) cp_async_4(dst, src); else cp_async_8(dst, src);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// FP32 with one compute warp: a second warp issues the cp.async copies of the
// next lines (a line's copies complete the stage's full mbarrier through
// cp.async.mbarrier.arrive.noinc; the compute warp frees the stage with an
// arrive on its empty mbarrier), so the compute warp issues no copies.  A
// clock64 trace had that issue at ~570 of ~1980 cycles per line.
template <typename T, int NW, bool USEPRE> struct ChainCopyWarp { static constexpr bool on = !USEPRE && NW == 1; };

template <typename T, int KPT, int NW, int NS, bool TRANS, bool USEPRE>
__global__ void __launch_bounds__(32 * NW + 32) k_line_chain2(ChainArgs<T> A) {
    typedef ChainSmem<T, KPT, NW, USEPRE> SM;
    constexpr bool CW = ChainCopyWarp<T, NW, USEPRE>::on;
    constexpr int VEC = SM::VEC, NV = KPT / VEC;
    typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V;
    if (A.skip && *A.skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *const stg = reinterpret_cast<T *>(smem_raw);
    __shared__ T sh[128];   // two buffers: the forward scan uses sh, the backward scan sh + 64
    const bool isY = blockIdx.x == 0;
    const Layout &lay = A.lay;
    const int L = lay.L;
    const Region &B = isY ? lay.R[2] : lay.R[1];
    const Region &C = lay.R[0], &I = lay.R[3];
    const int nlines = isY ? lay.R[2].mx : lay.R[1].my;
    const int tid = threadIdx.x, nthr = 32 * NW;
    const int e0 = tid * KPT;
    const T *const cpl = TRANS ? (isY ? A.wET : A.wNT) : (isY ? A.wE : A.wN);
    const T *const bcpl = isY ? A.wN : A.wE;
    const int owner = (L - 1) / KPT;   // the thread that owns the last node
    __shared__ __align__(8) unsigned long long fullb[NS], emptyb[NS];
    __shared__ unsigned abort_flag;
    if (tid == 0) {
        for (int q = 0; q < NS; q++) {
            mbar_init(&fullb[q], CW ? 32 : 1);   // copy warp: one arrival per lane and line
            mbar_init(&emptyb[q], 1);
        }
        abort_flag = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();

    if constexpr (CW) {
        if (tid >= 32 * NW) {   // ---- copy warp ----
            const int lane = tid & 31;
            for (int li = 0; li < nlines; li++) {
                const int q = li % NS, u = li / NS;
                if (u > 0) {   // the compute warp has read the line that used this stage before
                    mbar_wait(&emptyb[q], (unsigned)(u - 1) & 1u, &abort_flag, A.err);
                    if (abort_flag) break;
                }
                const int line = TRANS ? li : nlines - 1 - li;
                const long long base = B.off + (long long)line * L;
                T *st = stg + (size_t)q * SM::stage_elems;
                for (int k = lane; k < L / VEC; k += 32) {
                    const int e = k * VEC, p = SM::at(e);
                    cp_async_16(st + p, A.v + base + e);
                    cp_async_16(st + SM::LPP + p, cpl + base + e);
                    cp_async_16(st + 2 * SM::LPP + p, A.lf + base + e);
                    cp_async_16(st + 3 * SM::LPP + p, A.lg + base + e);
                    cp_async_16(st + 4 * SM::LPP + p, A.lh + base + e);
                }
                if (!TRANS && lane == 31) {   // boundary term of the last node: coupling * z_I
                    const long long pi = isY ? I.addr(line, 0) : I.addr(0, line);
                    cp_async_word(st + 5 * SM::LPP + SM::PRE, bcpl + base + (L - 1));
                    cp_async_word(st + 5 * SM::LPP + SM::PRE + 1, A.z + pi);
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&fullb[q])) : "memory");
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy lands after the CTA exits
            return;
        }
    }

    // line li's data into stage li % NS; every thread commits one (possibly
    // empty) cp.async group per line
    auto issue = [&](int li) {
        if (li < nlines) {
            const int line = TRANS ? li : nlines - 1 - li;
            const long long base = B.off + (long long)line * L;
            T *st = stg + (size_t)(li % NS) * SM::stage_elems;
            if constexpr (USEPRE) {
                if (tid == 0) {
                    unsigned long long *bar = &fullb[li % NS];
                    const unsigned lb = (unsigned)(L * sizeof(T));
                    mbar_arrive_expect_tx(bar, 5u * lb + (unsigned)(SM::PRE * sizeof(T)));
                    bulk_g2s(st, A.v + base, lb, bar);
                    bulk_g2s(st + SM::LPP, cpl + base, lb, bar);
                    bulk_g2s(st + 2 * SM::LPP, A.lf + base, lb, bar);
                    bulk_g2s(st + 3 * SM::LPP, A.lg + base, lb, bar);
                    bulk_g2s(st + 4 * SM::LPP, A.lh + base, lb, bar);
                    // this line's scan multipliers: 14 values per thread, [k][thread]
                    bulk_g2s(st + 5 * SM::LPP, A.pre + (size_t)(blockIdx.x * A.nlmax + line) * SM::PRE,
                             (unsigned)(SM::PRE * sizeof(T)), bar);
                }
            } else {
                for (int k = tid; k < L / VEC; k += nthr) {
                    const int e = k * VEC, p = SM::at(e);
                    cp_async_16(st + p, A.v + base + e);
                    cp_async_16(st + SM::LPP + p, cpl + base + e);
                    cp_async_16(st + 2 * SM::LPP + p, A.lf + base + e);
                    cp_async_16(st + 3 * SM::LPP + p, A.lg + base + e);
                    cp_async_16(st + 4 * SM::LPP + p, A.lh + base + e);
                }
            }
            if (!TRANS && tid == owner) {   // boundary term of the last node: coupling * z_I
                const long long pi = isY ? I.addr(line, 0) : I.addr(0, line);
                cp_async_word(st + 5 * SM::LPP + SM::PRE, bcpl + base + (L - 1));
                cp_async_word(st + 5 * SM::LPP + SM::PRE + 1, A.z + pi);
            }
        }
        cp_async_commit();
    };

    T zp[KPT], al[KPT], mu[KPT], y[KPT];
#pragma unroll
    for (int q = 0; q < KPT; q++) {   // transposed chain: the first line couples to C
        const int e = e0 + q;
        zp[q] = (TRANS && e < L && nlines > 0) ? A.z[isY ? C.addr(L - 1, e) : C.addr(e, L - 1)] : T(0);
    }
    if (!CW)
        for (int li = 0; li < NS - 1; li++) issue(li);
    for (int li = 0; li < nlines; li++) {
        // Stage (li - 1) % NS is refilled here: every thread read it before the
        // previous line's scans, whose barriers (NW > 1) or shuffles (one warp)
        // thread 0 has passed.
        if (USEPRE && NW == 1) __syncwarp();
        if (!CW) issue(li + NS - 1);
        if constexpr (CW) {
            if (!abort_flag) mbar_wait(&fullb[li % NS], (unsigned)(li / NS) & 1u, &abort_flag, A.err);
        } else if constexpr (USEPRE) {
            if (!abort_flag) mbar_wait(&fullb[li % NS], (unsigned)(li / NS) & 1u, &abort_flag, A.err);
            cp_async_wait<NS - 1>();     // the owner's boundary term of line li
        } else {
            cp_async_wait<NS - 1>();     // this thread's copies of line li have landed
            if (NW == 1) __syncwarp(); else __syncthreads();   // and every other thread's
        }
        const T *st = stg + (size_t)(li % NS) * SM::stage_elems;
        const int line = TRANS ? li : nlines - 1 - li;
        const long long base = B.off + (long long)line * L;
        T vv[KPT], cc[KPT], ff[KPT], g[KPT], hh[KPT];
        const int p0 = tid * SM::SEG;
#pragma unroll
        for (int r = 0; r < NV; r++) {
            const int p = p0 + r * VEC;
            *reinterpret_cast<V *>(vv + r * VEC) = *reinterpret_cast<const V *>(st + p);
            *reinterpret_cast<V *>(cc + r * VEC) = *reinterpret_cast<const V *>(st + SM::LPP + p);
            *reinterpret_cast<V *>(ff + r * VEC) = *reinterpret_cast<const V *>(st + 2 * SM::LPP + p);
            *reinterpret_cast<V *>(g + r * VEC) = *reinterpret_cast<const V *>(st + 3 * SM::LPP + p);
            *reinterpret_cast<V *>(hh + r * VEC) = *reinterpret_cast<const V *>(st + 4 * SM::LPP + p);
        }
        T bval = T(0);
        if (!TRANS && tid == owner) bval = st[5 * SM::LPP + SM::PRE] * st[5 * SM::LPP + SM::PRE + 1];
        if constexpr (CW) {   // stage read: the copy warp may refill it
            __syncwarp();
            if (tid == 0) mbar_arrive(&emptyb[li % NS]);
        }
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int e = e0 + q;
            if (e < L) {
                T d = vv[q] - cc[q] * zp[q];
                if (!TRANS && e == L - 1) d -= bval;
                al[q] = d;
                mu[q] = ff[q];
            } else {
                al[q] = T(0); mu[q] = T(1); g[q] = T(0); hh[q] = T(1);
            }
        }
        if constexpr (USEPRE) {
            T pf[7], pbk[7];
            const T *spre = st + 5 * SM::LPP;
#pragma unroll
            for (int k = 0; k < 7; k++) {
                pf[k] = spre[k * nthr + tid];
                pbk[k] = spre[(7 + k) * nthr + tid];
            }
            block_affine_scan_pre<T, KPT, false>(al, mu, pf, y, sh);
#pragma unroll
            for (int q = 0; q < KPT; q++) { al[q] = g[q] * y[q]; mu[q] = hh[q]; }
            block_affine_scan_pre<T, KPT, true>(al, mu, pbk, zp, sh + 64);
        } else {
            block_affine_scan<T, KPT, false>(al, mu, y, sh, NW);
#pragma unroll
            for (int q = 0; q < KPT; q++) { al[q] = g[q] * y[q]; mu[q] = hh[q]; }
            block_affine_scan<T, KPT, true>(al, mu, zp, sh, NW);
        }
#pragma unroll
        for (int r = 0; r < NV; r++)
            if (e0 + r * VEC < L) *reinterpret_cast<V *>(A.z + base + e0 + r * VEC) = *reinterpret_cast<const V *>(zp + r * VEC);
    }
    cp_async_wait<0>();
}

// Chain configuration (elements per thread, warps, stages) by line length
// and precision, shared by the launch and the multiplier precomputation.
template <int KPT_, int NW_, int NS_>
struct ChainCfg { static constexpr int KPT = KPT_, NW = NW_, NS = NS_; };
template <typename T, typename F>
static int with_chain_cfg(int L, F &&f) {
    if constexpr (sizeof(T) == 4) {
        if (L <= 512) return f(ChainCfg<16, 1, 8>{});
        if (L <= 1024) return f(ChainCfg<16, 2, 6>{});
        return f(ChainCfg<16, 4, 3>{});
    } else {
        if (L <= 512) return f(ChainCfg<4, 4, 4>{});
        if (L <= 1024) return f(ChainCfg<8, 4, 3>{});
        return f(ChainCfg<16, 4, 2>{});
    }
}
static bool chain2_applies(const blp_handle *h, size_t elem) {
    return h->L <= 2048 && (h->L * elem) % 16 == 0 && (h->lay.R[1].off * elem) % 16 == 0 &&
           (h->lay.R[2].off * elem) % 16 == 0;
}

// Setup: the scan multipliers of every line of both blocks, both scans, for
// the forward (lf, lh) or transposed (lfT, lhT) chain.  One CTA per line.
template <typename T, int KPT, int NW, bool TRANS>
__global__ void __launch_bounds__(32 * NW) k_chain_pre(Layout lay, const T *__restrict__ lf, const T *__restrict__ lh,
                                                       T *__restrict__ out, int nlmax) {
    const bool isY = blockIdx.y == 0;
    const int L = lay.L;
    const Region &B = isY ? lay.R[2] : lay.R[1];
    const int nlines = isY ? lay.R[2].mx : lay.R[1].my;
    const int line = blockIdx.x;
    if (line >= nlines) return;
    const long long base = B.off + (long long)line * L;
    const int tid = threadIdx.x, nthr = 32 * NW, e0 = tid * KPT;
    T mf[KPT], mh[KPT], p0[7], p1[7];
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = e0 + q;
        mf[q] = e < L ? lf[base + e] : T(1);
        mh[q] = e < L ? lh[base + e] : T(1);
    }
    scan_multipliers<T, KPT, false>(mf, p0);
    scan_multipliers<T, KPT, true>(mh, p1);
    T *o = out + (size_t)(blockIdx.y * nlmax + line) * (14 * nthr);
#pragma unroll
    for (int k = 0; k < 7; k++) {
        o[k * nthr + tid] = p0[k];
        o[(7 + k) * nthr + tid] = p1[k];
    }
}

template <typename T>
static int chain_pre_one(blp_handle *h, Coefs<T> &c) {
    if (!chain2_applies(h, sizeof(T))) return BLP_OK;
    const int nlmax = std::max(h->lay.R[2].mx, h->lay.R[1].my);
    return with_chain_cfg<T>(h->L, [&](auto cfg) -> int {
        using C = decltype(cfg);
        const size_t n = (size_t)2 * nlmax * 14 * 32 * C::NW;
        int rc;
        void *p = nullptr, *q = nullptr;
        if ((rc = blp_internal_alloc(h, &p, sizeof(T) * n))) return rc;
        c.cpre = static_cast<T *>(p);
        if ((rc = blp_internal_alloc(h, &q, sizeof(T) * n))) return rc;
        c.cpreT = static_cast<T *>(q);
        CUDA_TRY(cudaMemsetAsync(c.cpre, 0, sizeof(T) * n, h->stream));
        CUDA_TRY(cudaMemsetAsync(c.cpreT, 0, sizeof(T) * n, h->stream));
        const dim3 grid(std::max(nlmax, 1), 2);
        k_chain_pre<T, C::KPT, C::NW, false><<<grid, 32 * C::NW, 0, h->stream>>>(h->lay, c.lf, c.lh, c.cpre, nlmax);
        LAUNCH_CHECK(h);
        k_chain_pre<T, C::KPT, C::NW, true><<<grid, 32 * C::NW, 0, h->stream>>>(h->lay, c.lfT, c.lhT, c.cpreT, nlmax);
        LAUNCH_CHECK(h);
        return BLP_OK;
    });
}

int blp_internal_chain_pre(blp_handle *h) { return chain_pre_one<double>(h, h->cd); }

// FP64 chains use the precomputed multipliers (the FP64 scans are bound by one
// SM's FP64 FMA rate); FP32 chains, bound by latency, form them on the fly.
template <typename T, int KPT, int NW, int NS, bool TRANS>
static bool chain2_attrs_once() {
    constexpr bool USEPRE = sizeof(T) == 8;
    static std::atomic<bool> attr_set{false};
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_line_chain2<T, KPT, NW, NS, TRANS, USEPRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 225 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        attr_set = true;
    }
    return true;
}

template <typename T, int KPT, int NW, int NS, bool TRANS>
static int launch_chain2(blp_handle *h, const ChainArgs<T> &a) {
    constexpr bool USEPRE = sizeof(T) == 8;
    constexpr size_t smem = NS * ChainSmem<T, KPT, NW, USEPRE>::stage;
    static_assert(smem <= 225 * 1024, "line-chain stages exceed the shared-memory budget");
    if (!chain2_attrs_once<T, KPT, NW, NS, TRANS>()) return BLP_ERR_CUDA;
    k_line_chain2<T, KPT, NW, NS, TRANS, USEPRE>
        <<<2, 32 * NW + (ChainCopyWarp<T, NW, USEPRE>::on ? 32 : 0), smem, h->stream>>>(a);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

template <typename T, bool TRANS>
static int launch_chains(blp_handle *h, const Coefs<T> &c, const T *v, T *z, const int *skip) {
    ChainArgs<T> a;
    a.lay = h->lay; a.v = v; a.z = z;
    a.wE = c.wE; a.wN = c.wN; a.wET = c.wET; a.wNT = c.wNT;
    a.lf = TRANS ? c.lfT : c.lf; a.lg = TRANS ? c.lgT : c.lg; a.lh = TRANS ? c.lhT : c.lh;
    a.pre = nullptr; a.nlmax = 0;
    a.skip = skip;
    a.err = h->err;
    int L = h->L;
    // per line node: v, coupling, three factors, z = 6 words
    ProfScope ps(h, KC_LINE_CHAIN, (double)(h->lay.R[1].size + h->lay.R[2].size) * sizeof(T) * 6);
    if (chain2_applies(h, sizeof(T)) && (sizeof(T) == 4 || (TRANS ? c.cpreT : c.cpre))) {
        a.pre = TRANS ? c.cpreT : c.cpre;
        a.nlmax = std::max(h->lay.R[2].mx, h->lay.R[1].my);
        return with_chain_cfg<T>(L, [&](auto cfg) -> int {
            using C = decltype(cfg);
            return launch_chain2<T, C::KPT, C::NW, C::NS, TRANS>(h, a);
        });
    } else if (L <= 2048) {
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

// Scaled fine residual of the restriction, one thread per fine node:
// rr = omega_f (b - A e) (forward) or b - A^T e (transposed), zero on the
// padding slots.
template <typename T, bool TRANS>
__global__ void k_mg_residual(Level<T> F, const T *__restrict__ bf, const T *__restrict__ ef, T *__restrict__ rr,
                              const int *skip) {
    if (skip && *skip) return;
    const Region &RF = F.R;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < RF.size; q += (long long)gridDim.x * blockDim.x) {
        int a, bb;
        if (!RF.coords(q, a, bb)) { rr[q] = T(0); continue; }
        const T r = level_residual<T, TRANS>(F, bf, ef, a, bb);
        rr[q] = TRANS ? r : r * F.omega[q];
    }
}

// Restriction b_c = omega_c^-1 P^T rr (forward) or P^T rr (transposed): the
// full-weighting stencil over the fine residuals around node (2A+1, 2B+1).
template <typename T, bool TRANS>
__global__ void k_mg_restrict(Level<T> F, const T *__restrict__ rr, Level<T> Cc, T *__restrict__ bc, T *__restrict__ ec,
                              const int *skip) {
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
                sum += wx * wy * rr[RF.addr(a, bb)];
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
// stall2 > 0 (FP32 iterations): also stop once a cycle leaves ||r||^2 above
// stall2 times the previous cycle's (red[2]).  An FP32 iterate's residual has
// a rounding floor near 2^-24 || |A| |e| ||, which on a fine, diffusion-
// dominated corner (eps N >> 1) lies above the 1e3 reduction; the V-cycle
// contracts by far more than stall2 per cycle until it reaches that floor.
// When the iteration stops, flags[3] keeps the largest cycle count so far;
// flags[4] counts the cycles run since the solve began.
// use_cond: inside a captured solve, the conditional of the WHILE node that
// repeats the cycles is set to "not done" (an error flag also ends it).
__global__ void k_corner_finish(double *partials, int nb, DevState *st, int mode, double red2, int maxc,
                                double stall2, cudaGraphConditionalHandle cond, int use_cond, const int *err) {
    if (st->flags[0] && mode == 1) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
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
            st->flags[4] += 1;
            if (s <= st->red[0] || st->flags[1] >= maxc || (stall2 > 0.0 && s > stall2 * st->red[2])) st->flags[0] = 1;
            if (st->flags[0]) atomicMax(&st->flags[3], st->flags[1]);
        }
        st->red[2] = s;
        if (use_cond) cudaGraphSetConditional(cond, (st->flags[0] || (err && *err)) ? 0 : 1);
    }
}

// the FP32 corner iteration stops when a cycle fails to halve the residual
template <typename T> constexpr double corner_stall2() { return sizeof(T) == 4 ? 0.25 : 0.0; }

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
    int *err;                         // bounded-wait failures (BLP_ERR_TIMEOUT)
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
    T *c0;   // scratch of the sweep's right-hand side (shared by all levels)
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

// The same sweep for levels up to 64 wide, without a barrier per diagonal.
// A CTA-parallel pass first forms c0 = b - (terms of the neighbours the sweep
// reaches later, still old: W and S forward, E and N transposed).  One warp
// then runs the wavefront with the new neighbour values in registers: the
// node's own column's last value (N forward, S transposed) and, through one
// shuffle, the adjacent lane's (E forward, W transposed).  Lane l owns column
// l (m <= 32) or columns 2l, 2l+1 (m <= 64); with two columns the second
// column's chain neighbour is the lane's own first column.  The node of
// column a handled at step t lies on row b = (2m-2-t) - a forward, t - a
// transposed; outside the level a lane carries 0.
template <typename T, bool TRANS>
__device__ __forceinline__ void coarse_gs_chain(const CLev<T> L) {
    const int m = L.m, n = m * m;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int a = k % m, bb = k / m;
        T s = L.b[k];
        if (!TRANS) {
            if (a > 0) s -= L.cw[k] * L.e[k - 1];
            if (bb > 0) s -= L.cs[k] * L.e[k - m];
        } else {
            if (a < m - 1) s -= L.ce[k] * L.e[k + 1];
            if (bb < m - 1) s -= L.cn[k] * L.e[k + m];
        }
        L.c0[k] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        // chain couplings: forward E (horizontal) and N (vertical), transposed W and S
        const T *__restrict__ ch = TRANS ? L.cw : L.ce;
        const T *__restrict__ cv = TRANS ? L.cs : L.cn;
        const T *__restrict__ c0 = L.c0;
        T *__restrict__ e = L.e;
        const int nst = 2 * m - 1;
        const int dk = TRANS ? m : -m;   // node index change per step along a column
        // column a is on the level during steps [lo(a), lo(a) + m - 1]: forward
        // from row m-1 at step m-1-a down to row 0, transposed from row 0 at step a
        auto first_step = [&](int a) { return TRANS ? a : m - 1 - a; };
        auto first_node = [&](int a) { return TRANS ? a : (m - 1) * m + a; };
        constexpr int G = 4;   // steps per group: their shared-memory loads are issued together
        if (m <= 32) {
            T z = T(0);
            const int a = lane;
            const bool live = a < m, headl = lane == (TRANS ? 0 : 31);
            const int lo = first_step(a);
            int k = first_node(a) - lo * dk;   // the (virtual) node index at step 0
            for (int t0 = 0; t0 < nst; t0 += G, k += G * dk) {
                T cc[G], cvv[G], chh[G];
                bool ok[G];
#pragma unroll
                for (int u = 0; u < G; u++) {
                    ok[u] = live && (unsigned)(t0 + u - lo) < (unsigned)m;
                    const int ku = k + u * dk;
                    cc[u] = ok[u] ? c0[ku] : T(0);
                    cvv[u] = ok[u] ? cv[ku] : T(0);
                    chh[u] = ok[u] && !headl ? ch[ku] : T(0);
                }
#pragma unroll
                for (int u = 0; u < G; u++) {
                    const T zh = TRANS ? __shfl_up_sync(FULL, z, 1) : __shfl_down_sync(FULL, z, 1);
                    T v = cc[u] - cvv[u] * z;
                    v = v - chh[u] * zh;
                    if (ok[u]) e[k + u * dk] = v;
                    z = ok[u] ? v : T(0);
                }
            }
        } else {
            // columns a0 = 2 lane, a1 = 2 lane + 1; z0, z1 their last values
            T z0 = T(0), z1 = T(0);
            const int a0 = 2 * lane, a1 = a0 + 1;
            const bool live0 = a0 < m, live1 = a1 < m, headl = lane == (TRANS ? 0 : 31);
            const int lo0 = first_step(a0), lo1 = first_step(a1);
            int k0 = first_node(a0) - lo0 * dk, k1 = first_node(a1) - lo1 * dk;
            for (int t0 = 0; t0 < nst; t0 += G, k0 += G * dk, k1 += G * dk) {
                T c0a[G], cva[G], cha[G], c0b[G], cvb[G], chb[G];
                bool oka[G], okb[G];
#pragma unroll
                for (int u = 0; u < G; u++) {
                    oka[u] = live0 && (unsigned)(t0 + u - lo0) < (unsigned)m;
                    okb[u] = live1 && (unsigned)(t0 + u - lo1) < (unsigned)m;
                    const int ka = k0 + u * dk, kb = k1 + u * dk;
                    c0a[u] = oka[u] ? c0[ka] : T(0);
                    cva[u] = oka[u] ? cv[ka] : T(0);
                    cha[u] = oka[u] && !(TRANS && headl) ? ch[ka] : T(0);
                    c0b[u] = okb[u] ? c0[kb] : T(0);
                    cvb[u] = okb[u] ? cv[kb] : T(0);
                    chb[u] = okb[u] && !(!TRANS && headl) ? ch[kb] : T(0);
                }
#pragma unroll
                for (int u = 0; u < G; u++) {
                    // forward: E of column a1 is the next lane's column a0; transposed: W of
                    // column a0 is the previous lane's column a1
                    const T zh = TRANS ? __shfl_up_sync(FULL, z1, 1) : __shfl_down_sync(FULL, z0, 1);
                    T v0, v1;
                    if (!TRANS) {
                        // (a1, b1): E = next lane's column a0, N = own z1
                        v1 = c0b[u] - cvb[u] * z1;
                        v1 = v1 - chb[u] * zh;
                        // (a0, b0 = b1 + 1): E = (a1, b1 + 1) = own z1 (last step), N = own z0
                        v0 = c0a[u] - cva[u] * z0;
                        v0 = v0 - cha[u] * z1;
                    } else {
                        // (a0, b0): W = previous lane's column a1, S = own z0
                        v0 = c0a[u] - cva[u] * z0;
                        v0 = v0 - cha[u] * zh;
                        // (a1, b1 = b0 - 1): W = (a0, b0 - 1) = own z0 (last step), S = own z1
                        v1 = c0b[u] - cvb[u] * z1;
                        v1 = v1 - chb[u] * z0;
                    }
                    if (oka[u]) e[k0 + u * dk] = v0;
                    if (okb[u]) e[k1 + u * dk] = v1;
                    z0 = oka[u] ? v0 : T(0);
                    z1 = okb[u] ? v1 : T(0);
                }
            }
        }
    }
    __syncthreads();
}

template <typename T, bool TRANS>
__device__ __forceinline__ void coarse_gs(const CLev<T> L) {
    if (L.m <= 64) {
        coarse_gs_chain<T, TRANS>(L);
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
    __shared__ CLev<T> LV[BLP_MAXLEV];   // level descriptors (one copy, not per thread)
    if (threadIdx.x == 0) {
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
        }
        for (int l = A.l0; l < A.nlev; l++) LV[l].c0 = p;   // sweep scratch, the size of level l0
    }
    // the static coefficients: one 1D bulk copy per array when every array
    // is a whole number of 16-byte units (then all offsets are aligned too),
    // else element by element below
    __shared__ __align__(8) unsigned long long cbar;
    bool bulk = true;
    for (int l = A.l0; l < A.nlev; l++) bulk = bulk && (A.m[l] * A.m[l] * (int)sizeof(T)) % 16 == 0;
    if (bulk && threadIdx.x == 0) {
        unsigned bytes = 0;
        for (int l = A.l0; l < A.nlev; l++) bytes += (TRANS ? 6u : 5u) * (unsigned)(A.m[l] * A.m[l] * sizeof(T));
        mbar_init(&cbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_arrive_expect_tx(&cbar, bytes);
        for (int l = A.l0; l < A.nlev; l++) {
            const int n = A.m[l] * A.m[l];
            const unsigned nb = (unsigned)(n * sizeof(T));
            const CLev<T> &L = LV[l];
            const T *nat = A.nat[l];
            const int q0 = TRANS ? 4 : 0;
            bulk_g2s(L.cw, nat + (long long)(q0 + 0) * n, nb, &cbar);
            bulk_g2s(L.ce, nat + (long long)(q0 + 1) * n, nb, &cbar);
            bulk_g2s(L.cs, nat + (long long)(q0 + 2) * n, nb, &cbar);
            bulk_g2s(L.cn, nat + (long long)(q0 + 3) * n, nb, &cbar);
            bulk_g2s(L.om, nat + (long long)8 * n, nb, &cbar);
            if (TRANS) bulk_g2s(L.wt, nat + (long long)9 * n, nb, &cbar);
        }
    }
    __syncthreads();
    if (!bulk) {
        for (int l = A.l0; l < A.nlev; l++) {
            const int n = A.m[l] * A.m[l];
            const CLev<T> L = LV[l];
            const T *__restrict__ nat = A.nat[l];
            const int q0 = TRANS ? 4 : 0;
            // four elements per thread in flight: the loads are issued before the stores
            for (int k0 = threadIdx.x; k0 < n; k0 += 4 * blockDim.x) {
                T v[4][6];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int k = k0 + u * blockDim.x;
                    if (k < n) {
                        v[u][0] = __ldg(nat + (long long)(q0 + 0) * n + k);
                        v[u][1] = __ldg(nat + (long long)(q0 + 1) * n + k);
                        v[u][2] = __ldg(nat + (long long)(q0 + 2) * n + k);
                        v[u][3] = __ldg(nat + (long long)(q0 + 3) * n + k);
                        v[u][4] = __ldg(nat + (long long)8 * n + k);
                        v[u][5] = TRANS ? __ldg(nat + (long long)9 * n + k) : T(0);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int k = k0 + u * blockDim.x;
                    if (k < n) {
                        L.cw[k] = v[u][0]; L.ce[k] = v[u][1]; L.cs[k] = v[u][2]; L.cn[k] = v[u][3];
                        L.om[k] = v[u][4];
                        if (TRANS) L.wt[k] = v[u][5];
                    }
                }
            }
        }
    }
    const int l0 = A.l0, last = A.nlev - 1, m0 = A.m[l0];
    const Region R0 = A.R0;
    for (int k0 = threadIdx.x; k0 < m0 * m0; k0 += 4 * blockDim.x) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int k = k0 + u * blockDim.x;
            if (k < m0 * m0) v[u] = __ldg(A.b_in + R0.addr(k % m0, k / m0));
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int k = k0 + u * blockDim.x;
            if (k < m0 * m0) { LV[l0].b[k] = v[u]; LV[l0].e[k] = T(0); }
        }
    }
    if (bulk) {   // the copies read valid memory and complete; the wait is bounded all the same
        long long it = 0;
        while (!mbar_try_wait(&cbar, 0u)) {
            if (++it > (BLP_SPIN_LIMIT >> 4)) {
                if (threadIdx.x == 0) atomicExch(A.err, BLP_ERR_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();

    auto vcycle = [&]() {
        for (int l = l0; l < last; l++) {
            const CLev<T> F = LV[l], Cc = LV[l + 1];
            const int m = F.m, mc = Cc.m;
            coarse_gs<T, TRANS>(F);
            // restriction of the residual: forward b_c = omega_c^-1 P^T omega_f r, transpose
            // b_c = P^T r; the (scaled) residual of every fine node once, into the scratch
            for (int k = threadIdx.x; k < m * m; k += blockDim.x) {
                T r = coarse_residual<T>(F, k % m, k / m);
                if (!TRANS) r *= F.om[k];
                F.c0[k] = r;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < mc * mc; q += blockDim.x) {
                const int a0 = 2 * (q % mc) + 1, b0 = 2 * (q / mc) + 1;
                T sum = T(0);
                for (int db = -1; db <= 1; db++) {
                    const int bb = b0 + db;
                    if (bb < 0 || bb >= m) continue;
                    for (int da = -1; da <= 1; da++) {
                        const int a = a0 + da;
                        if (a < 0 || a >= m) continue;
                        sum += (da == 0 ? T(1) : T(0.5)) * (db == 0 ? T(1) : T(0.5)) * F.c0[bb * m + a];
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
    return b + sizeof(T) * (size_t)H.lev[l0].R.mx * H.lev[l0].R.mx;   // + the sweep scratch
}

// first level handled by the fused coarse kernel (-1: none)
template <typename T>
static int coarse_start(const Hierarchy<T> &H) {
    for (int l = 0; l < H.nlev; l++)
        if (H.lev[l].nat && coarse_smem(H, l) <= 200 * 1024) return l;
    return -1;
}

template <typename T, bool TRANS>
static bool coarse_attrs_once() {
    static std::atomic<bool> attr{false};
    if (!attr) {
        // dynamic bytes this kernel ever asks for (coarse_start caps them at 200 KB); it also
        // has a little static shared memory, so the opt-in maximum itself would be rejected
        if (cudaFuncSetAttribute(k_mg_coarse<T, TRANS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        attr = true;
    }
    return true;
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
    a.st = h->dev; a.skip = skip; a.err = h->err;
    const size_t smem = coarse_smem(H, l0);
    if (!coarse_attrs_once<T, TRANS>()) return BLP_ERR_CUDA;
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
            // fine b, e, 4 couplings, omega read and the residual written; then
            // the residual read and coarse b (and e) written
            ProfScope ps(h, KC_MG_RESTRICT, ((double)Lv.R.mx * Lv.R.my * 9 + (double)Cn.R.mx * Cn.R.my * 2) * sizeof(T));
            k_mg_residual<T, TRANS><<<grid_for(Lv.R.size, 256), 256, 0, h->stream>>>(Lv, b, Lv.e[cur[l]], Lv.beta, skip);
            LAUNCH_CHECK(h);
            k_mg_restrict<T, TRANS><<<grid_for(Cn.R.size, 256), 256, 0, h->stream>>>(Lv, Lv.beta, Cn, Cn.b,
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
// e = 0; the result is left in the returned level-0 buffer.  The iteration
// is enqueued in two parts: corner_front (the initial norm and a batch of
// cycles, each ending with the stopping test that sets the device skip flag
// -- no host synchronisation, so it can be captured in a graph) and
// corner_rest (read the flag; more cycles while the test fails).
template <typename T, bool TRANS>
static int corner_more(blp_handle *h, const T *b0, Cycler<T, TRANS> &cy, int count, int *enq) {
    Hierarchy<T> &H = hier_of<T>(h);
    Level<T> &L0 = H.lev[0];
    const int nb = BLP_RED_BLOCKS;
    const double red2 = h->p.corner_reduction * h->p.corner_reduction;
    int *done = h->dev->flags;
    for (int c = 0; c < count && *enq < h->p.corner_max_cycles; c++, (*enq)++) {
        int rc = cy.vcycle(0);
        if (rc) return rc;
        ProfScope ps(h, KC_CORNER_NORM, (double)L0.R.mx * L0.R.my * 7 * sizeof(T));
        k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[cy.cur[0]], 1, h->partials, done);
        LAUNCH_CHECK(h);
        k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 1, red2, h->p.corner_max_cycles,
                                                 corner_stall2<T>(), 0, 0, nullptr);
        LAUNCH_CHECK(h);
    }
    return BLP_OK;
}

template <typename T, bool TRANS>
static int corner_front(blp_handle *h, const T *b0, Cycler<T, TRANS> &cy, int batch, int *enq) {
    Hierarchy<T> &H = hier_of<T>(h);
    Level<T> &L0 = H.lev[0];
    for (int l = 0; l < H.nlev; l++) { cy.cur[l] = 0; cy.zero[l] = false; }
    cy.zero[0] = true;
    CUDA_TRY(cudaMemsetAsync(L0.e[0], 0, sizeof(T) * L0.R.size, h->stream));
    const int nb = BLP_RED_BLOCKS;
    const double red2 = h->p.corner_reduction * h->p.corner_reduction;
    int *done = h->dev->flags;   // flags[0]
    cy.skip = nullptr;
    {
        ProfScope ps(h, KC_CORNER_NORM, (double)L0.R.mx * L0.R.my * 2 * sizeof(T));
        k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[0], 0, h->partials, nullptr);
        LAUNCH_CHECK(h);
        k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 0, red2, h->p.corner_max_cycles,
                                                 corner_stall2<T>(), 0, 0, nullptr);
        LAUNCH_CHECK(h);
    }
    cy.skip = done;
    *enq = 0;
    return corner_more(h, b0, cy, batch, enq);
}

template <typename T, bool TRANS>
static int corner_rest(blp_handle *h, const T *b0, Cycler<T, TRANS> &cy, int *enq, int *cycles) {
    for (;;) {
        CUDA_TRY(cudaMemcpyAsync(h->host_state, h->dev, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (h->host_state->flags[0] || *enq >= h->p.corner_max_cycles) break;
        int rc = corner_more(h, b0, cy, 2, enq);
        if (rc) return rc;
    }
    *cycles = h->host_state->flags[1];
    h->last_cycles = *cycles + 1;
    return BLP_OK;
}

// Inside a captured solve: the first cycle (from e = 0), then a WHILE node
// whose body is one more cycle with its stopping test; every test sets the
// node's conditional, so the cycles repeat on the device until the test
// passes or the cycle cap is reached.  One cycle leaves every level's
// iterate in the buffer it started in, so all cycles are the same body.
template <typename T, bool TRANS>
static int corner_solve_captured(blp_handle *h, const T *b0, Cycler<T, TRANS> &cy, T **result) {
    Hierarchy<T> &H = hier_of<T>(h);
    Level<T> &L0 = H.lev[0];
    const int nb = BLP_RED_BLOCKS;
    const double red2 = h->p.corner_reduction * h->p.corner_reduction;
    int *done = h->dev->flags;
    int rc;
    for (int l = 0; l < H.nlev; l++) { cy.cur[l] = 0; cy.zero[l] = false; }
    cy.zero[0] = true;
    CUDA_TRY(cudaMemsetAsync(L0.e[0], 0, sizeof(T) * L0.R.size, h->stream));
    cy.skip = nullptr;
    k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[0], 0, h->partials, nullptr);
    LAUNCH_CHECK(h);
    k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 0, red2, h->p.corner_max_cycles,
                                             corner_stall2<T>(), 0, 0, nullptr);
    LAUNCH_CHECK(h);
    cy.skip = done;
    cudaGraphConditionalHandle cond;
    if ((rc = cap_handle(h, 0, &cond))) return rc;
    auto cycle = [&]() -> int {
        int r2 = cy.vcycle(0);
        if (r2) return r2;
        k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[cy.cur[0]], 1, h->partials, done);
        LAUNCH_CHECK(h);
        k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 1, red2, h->p.corner_max_cycles,
                                                 corner_stall2<T>(), cond, 1, h->err);
        LAUNCH_CHECK(h);
        return BLP_OK;
    };
    if ((rc = cycle())) return rc;
    int cur0[BLP_MAXLEV];
    for (int l = 0; l < H.nlev; l++) cur0[l] = cy.cur[l];
    if ((rc = cap_begin(h, cond, cudaGraphCondTypeWhile))) return rc;
    const long long l0 = h->launches;
    rc = cycle();
    h->corner_body_launches = h->launches - l0;
    const int rc2 = cap_end(h);
    if (rc) return rc;
    if (rc2) return rc2;
    for (int l = 0; l < H.nlev; l++)
        if (cy.cur[l] != cur0[l]) return BLP_ERR_ARG;   // a cycle must end where it began
    *result = L0.e[cy.cur[0]];
    return BLP_OK;
}

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
    Level<T> &L0 = H.lev[0];
    const int fixed = h->p.corner_fixed_cycles;
    int cycles = 0;
    if (fixed > 0) {
        for (int l = 0; l < H.nlev; l++) { cy.cur[l] = 0; cy.zero[l] = false; }
        cy.zero[0] = true;
        CUDA_TRY(cudaMemsetAsync(L0.e[0], 0, sizeof(T) * L0.R.size, h->stream));
        cy.skip = nullptr;
        for (int c = 0; c < fixed; c++) { int rc = cy.vcycle(0); if (rc) return rc; }
        cycles = fixed;
    } else if (h->capturing) {
        int rc = corner_solve_captured<T, TRANS>(h, b0, cy, result);
        if (cycles_out) *cycles_out = -1;
        return rc;
    } else {
        int enq = 0, rc;
        const int batch = std::max(2, std::min(h->last_cycles > 0 ? h->last_cycles : 6, h->p.corner_max_cycles));
        if ((rc = corner_front<T, TRANS>(h, b0, cy, batch, &enq))) return rc;
        if ((rc = corner_rest<T, TRANS>(h, b0, cy, &enq, &cycles))) return rc;
    }
    *result = L0.e[cy.cur[0]];
    if (cycles_out) *cycles_out = cycles;
    return BLP_OK;
}

// The front of one application -- for the forward map the interior sweep,
// the line chains, the corner right-hand side and the corner_front batch;
// for the transposed map the corner_front batch -- is enqueued with no host
// synchronisation.  On a capturable stream it is captured once per
// (precision, direction, corner batch) as a CUDA graph that reads and
// writes two fixed buffers of the handle, and replayed: two copies and one
// launch instead of about a hundred launches.
template <typename T>
static int precond_front(blp_handle *h, const T *v, T *z, int trans, Cycler<T, false> &cf, Cycler<T, true> &ct,
                         int batch, int *enq) {
    Coefs<T> &c = coefs_of<T>(h);
    Hierarchy<T> &H = hier_of<T>(h);
    const Layout &lay = h->lay;
    const Region &C = lay.R[0];
    int rc;
    if (!trans) {
        DtsArgs<T> a;
        a.R = lay.R[3]; a.beta = v; a.pair = c.pF; a.out = z;
        a.bnd = nullptr; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, false>(h, a, KC_DTS_INTERIOR))) return rc;
        if ((rc = launch_chains<T, false>(h, c, v, z, nullptr))) return rc;
        T *b0 = H.lev[0].b;
        {
            ProfScope ps(h, KC_LAYOUT);
            k_corner_rhs<T><<<grid_for(C.size, 256), 256, 0, h->stream>>>(lay, v, z, c.wE, c.wN, b0, nullptr);
            LAUNCH_CHECK(h);
        }
        return corner_front<T, false>(h, b0, cf, batch, enq);
    }
    return corner_front<T, true>(h, v + C.off, ct, batch, enq);
}

template <typename T>
static int precond_graph(blp_handle *h, const T *v_in, T *z_out, int trans, int *cycles) {
    Hierarchy<T> &H = hier_of<T>(h);
    const Layout &lay = h->lay;
    const Region &C = lay.R[0];
    const int prec = sizeof(T) == 4 ? 1 : 0;
    const size_t bytes = sizeof(T) * (size_t)lay.npad;
    int rc;
    if (!h->gv[prec]) {
        if ((rc = blp_internal_alloc(h, &h->gv[prec], bytes))) return rc;
        if ((rc = blp_internal_alloc(h, &h->gz[prec], bytes))) return rc;
        CUDA_TRY(cudaMemsetAsync(h->gv[prec], 0, bytes, h->stream));
        CUDA_TRY(cudaMemsetAsync(h->gz[prec], 0, bytes, h->stream));
    }
    const T *v = static_cast<const T *>(h->gv[prec]);
    T *z = static_cast<T *>(h->gz[prec]);
    CUDA_TRY(cudaMemcpyAsync(h->gv[prec], v_in, bytes, cudaMemcpyDeviceToDevice, h->stream));
    const int batch = std::max(2, std::min(h->last_cycles > 0 ? h->last_cycles : 6, h->p.corner_max_cycles));
    Cycler<T, false> cf;
    Cycler<T, true> ct;
    cf.h = ct.h = h; cf.H = ct.H = &H; cf.l0c = ct.l0c = coarse_start(H);
    cf.b0 = H.lev[0].b;
    ct.b0 = v + C.off;
    blp_handle::PrecGraph *G = nullptr;
    for (auto &g : h->graphs)
        if (g.trans == trans && g.prec == prec && g.batch == batch) { G = &g; break; }
    if (!G) {
        blp_handle::PrecGraph g;
        memset(&g, 0, sizeof(g));
        g.trans = trans; g.prec = prec; g.batch = batch;
        const long long l0 = h->launches;
        CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int enq = 0;
        rc = precond_front<T>(h, v, z, trans, cf, ct, batch, &enq);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (rc != BLP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            h->use_graphs = false;
            return rc != BLP_OK ? rc : BLP_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->use_graphs = false;
            return BLP_ERR_CUDA;
        }
        g.nlaunch = h->launches - l0;
        h->launches = l0;
        g.enq = enq;
        for (int l = 0; l < BLP_MAXLEV; l++) {
            g.cur[l] = trans ? ct.cur[l] : cf.cur[l];
            g.zero[l] = trans ? ct.zero[l] : cf.zero[l];
        }
        h->graphs.push_back(g);
        G = &h->graphs.back();
    }
    CUDA_TRY(cudaGraphLaunch(G->exec, h->stream));
    h->launches += G->nlaunch;
    // continue the corner iteration from the captured state if its test failed
    int enq = G->enq, cyc = 0;
    int *done = h->dev->flags;
    T *e = nullptr;
    if (!trans) {
        for (int l = 0; l < BLP_MAXLEV; l++) { cf.cur[l] = G->cur[l]; cf.zero[l] = G->zero[l]; }
        cf.skip = done;
        if ((rc = corner_rest<T, false>(h, cf.b0, cf, &enq, &cyc))) return rc;
        e = H.lev[0].e[cf.cur[0]];
    } else {
        for (int l = 0; l < BLP_MAXLEV; l++) { ct.cur[l] = G->cur[l]; ct.zero[l] = G->zero[l]; }
        ct.skip = done;
        if ((rc = corner_rest<T, true>(h, ct.b0, ct, &enq, &cyc))) return rc;
        e = H.lev[0].e[ct.cur[0]];
    }
    {
        ProfScope ps(h, KC_LAYOUT);
        CUDA_TRY(cudaMemcpyAsync(z + C.off, e, sizeof(T) * C.size, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (trans) {
        Coefs<T> &c = coefs_of<T>(h);
        if ((rc = launch_chains<T, true>(h, c, v, z, nullptr))) return rc;
        DtsArgs<T> a;
        a.R = lay.R[3]; a.beta = v; a.pair = c.pR; a.out = z;
        a.bnd = z; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, true>(h, a, KC_DTS_INTERIOR))) return rc;
    }
    CUDA_TRY(cudaMemcpyAsync(z_out, z, bytes, cudaMemcpyDeviceToDevice, h->stream));
    if (cycles) *cycles = cyc;
    return BLP_OK;
}

template <typename T>
int precond_apply(blp_handle *h, const T *v, T *z, int trans, int *cycles) {
    const int prec = sizeof(T) == 4 ? 1 : 0;
    if (h->semi && trans) return BLP_ERR_ARG;   // the parabolic-layer corner cycle is forward only
    if (h->use_graphs && h->warm[prec][trans ? 1 : 0] && h->stream != 0 && !h->prof.on && !h->capturing &&
        h->p.corner_fixed_cycles <= 0 && coarse_start(hier_of<T>(h)) > 0 && !h->semi)
        return precond_graph<T>(h, v, z, trans, cycles);
    if (!h->capturing) h->warm[prec][trans ? 1 : 0] = true;   // the first application runs eagerly (kernel attributes set outside any capture)
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
        if (h->semi) return semi_corner_solve<T>(h, b0, z + C.off, cycles);   // Sec. 3.2, parabolic case
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

// Kernel attributes of everything one application can launch, set before a
// whole-solve capture begins (no attribute is set inside a capture).
template <typename T>
int precond_capture_prepare(blp_handle *h) {
    if (!dts_attrs_all<T>() || !coarse_attrs_once<T, false>() || !coarse_attrs_once<T, true>()) return BLP_ERR_CUDA;
    if (chain2_applies(h, sizeof(T))) {
        const bool ok = with_chain_cfg<T>(h->L, [&](auto cfg) -> int {
            using C = decltype(cfg);
            return chain2_attrs_once<T, C::KPT, C::NW, C::NS, false>() && chain2_attrs_once<T, C::KPT, C::NW, C::NS, true>();
        });
        if (!ok) return BLP_ERR_CUDA;
    }
    return BLP_OK;
}
template int precond_capture_prepare<double>(blp_handle *);
template int precond_capture_prepare<float>(blp_handle *);
