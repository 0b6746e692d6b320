// blp_dts.cuh -- the wavefront kernel of the boundary-layer preconditioner
// (the downstream triangular solves of Sec. 3.1 and the Gauss-Seidel
// smoother of Sec. 3.2), its launch, and the self-check of its bounded
// waits.  Included once, by blp_precond.cu.
#pragma once
#include "blp_common.cuh"
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

#ifndef FULL
#define FULL 0xffffffffu
#endif

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
// Lane l of the warp that owns a 32-column strip handles column 32s+l and,
// at step t, diagonal d = t (forward) or D-1-t (reversed), so each step
// reads 32 consecutive words of beta and of the packed (cH, cV) pairs; those
// arrive by bulk copies several chunks ahead, so memory latency stays off the
// recurrence, whose step is one shuffle and two FMAs.  The lane next to the
// previous strip ("head") takes that strip's boundary column from a ring in
// shared memory filled by the warp that processed it.
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

// bounded wait on the mbarrier phase of this warp's own bulk copies
// (BLP_ERR_TIMEOUT instead of a hang).  It does not stop at the abort flag:
// the copies read valid memory and always complete, and waiting for them
// keeps any copy from landing after the CTA has exited.
__device__ __forceinline__ void mbar_wait(unsigned long long *bar, unsigned parity, volatile unsigned *abort_flag, int *err) {
    unsigned ready;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ready) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (ready) return;   // usually complete already
    long long n = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++n > (BLP_SPIN_LIMIT >> 4)) {
            *abort_flag = 1u;
            atomicExch(err, BLP_ERR_TIMEOUT);
            return;
        }
    }
}

// Shared-memory carve-up of one CTA: WC compute warps plus one copy warp.
// Per compute warp: NST stages of CH diagonals of (cH, cV) pairs (T2) and
// beta (T); an input ring of NSL slots of RS boundary values (DtsRing); full and
// empty mbarriers per stage; one mbarrier per ring slot.  Then per compute
// warp the count of ring slots its successor has released, the wave counter
// and the abort flag.
// Hand-off granularity: boundary values per ring slot, and ring slots per
// compute warp.  FP32 hands off whole chunks: its 34-cycle steps make the
// per-slot wait, re-arm and stores cost more than a shorter lag between
// strips saves (measured: 8-value slots made the 512^2 sweep 30% slower).
// FP64 steps take ~220 cycles, and 8-value slots shorten the lag (measured
// 3% faster).
template <typename T, int CH>
struct DtsRing {
    static constexpr int RS = sizeof(T) == 4 ? CH : (CH < 8 ? CH : 8);
    static constexpr int NSL = RS >= 16 ? 16 : 32;
};

template <typename T, int CH>
struct DtsSmem {
    typedef typename Vec2T<T>::type T2;
    static constexpr size_t stage_pairs = (size_t)CH * 32 * sizeof(T2);
    static constexpr size_t stage_beta = (size_t)CH * 32 * sizeof(T);
    static constexpr size_t stage = stage_pairs + stage_beta;
    static constexpr int NSL = DtsRing<T, CH>::NSL;
    static constexpr size_t ring = (size_t)NSL * DtsRing<T, CH>::RS * sizeof(T);
    static size_t bytes(int WC, int NST) {
        return (size_t)WC * (NST * stage + ring + 16 * (size_t)NST + 8 * (size_t)NSL + 4) + 64;
    }
};

// --- distributed shared memory and mbarrier helpers (inline PTX) -----------
__device__ __forceinline__ unsigned mapa_u32(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// RS boundary values (from a register array, compile-time offsets) into a
// ring slot, as asynchronous vector stores completing the slot's mbarrier
template <int RS>
__device__ __forceinline__ void st_async_rs(unsigned addr, const float *v, unsigned bar) {
#pragma unroll
    for (int i = 0; i < RS / 4; i++)
        asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];\n"
                     ::"r"(addr + 16 * i), "r"(__float_as_uint(v[4 * i])), "r"(__float_as_uint(v[4 * i + 1])),
                     "r"(__float_as_uint(v[4 * i + 2])), "r"(__float_as_uint(v[4 * i + 3])), "r"(bar) : "memory");
}
template <int RS>
__device__ __forceinline__ void st_async_rs(unsigned addr, const double *v, unsigned bar) {
#pragma unroll
    for (int i = 0; i < RS / 2; i++)
        asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];\n"
                     ::"r"(addr + 16 * i), "l"(__double_as_longlong(v[2 * i])), "l"(__double_as_longlong(v[2 * i + 1])),
                     "r"(bar) : "memory");
}
// one 16-byte piece of a ring slot (4 FP32 / 2 FP64 values), stored only
// where `on` is set, so a warp issues it without branching
__device__ __forceinline__ void st_async_16(bool on, unsigned addr, const float *v, unsigned bar) {
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %6, 0;\n"
                 " @q st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];\n}\n"
                 ::"r"(addr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(bar), "r"((unsigned)on) : "memory");
}
__device__ __forceinline__ void st_async_16(bool on, unsigned addr, const double *v, unsigned bar) {
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                 " @q st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];\n}\n"
                 ::"r"(addr), "l"(__double_as_longlong(v[0])), "l"(__double_as_longlong(v[1])), "r"(bar),
                 "r"((unsigned)on) : "memory");
}
__device__ __forceinline__ void st_relaxed_cluster(unsigned addr, unsigned v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_cluster(unsigned addr, unsigned v) {
    asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cluster(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];\n" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait for a ring slot filled by a peer (stops at the abort flag)
__device__ __forceinline__ bool mbar_test_wait_cluster(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_wait_cluster(unsigned long long *bar, unsigned parity, volatile unsigned *abort_flag,
                                                  int *err, long long limit = BLP_SPIN_LIMIT >> 4) {
    if (mbar_test_wait_cluster(bar, parity)) return;   // usually complete already
    long long n = 0;
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (*abort_flag) return;
        if (++n > limit) {
            *abort_flag = 1u;
            atomicExch(err, BLP_ERR_TIMEOUT);
            return;
        }
    }
}
// bounded wait until the local counter *ctr (written by a peer) >= target;
// returns the last value read
__device__ __forceinline__ int wait_counter(const unsigned *ctr, int target, volatile unsigned *abort_flag, int *err,
                                            long long limit = BLP_SPIN_LIMIT) {
    long long n = 0;
    int v;
    while ((v = (int)ld_acquire_cluster(ctr)) < target) {
        if (*abort_flag) return v;
        if (++n > limit) {
            *abort_flag = 1u;
            atomicExch(err, BLP_ERR_TIMEOUT);
            return v;
        }
    }
    return v;
}

// The kernel runs as one thread-block cluster of CL CTAs, each with WC
// compute warps and one copy warp (W = CL*WC compute warps; global compute
// warp g = rank*WC + w).  Strips go to compute warps in waves of W.
//  - The copy warp keeps NST stages per compute warp filled with bulk
//    copies (full / empty mbarriers), so compute warps never issue copies.
//  - Inside a wave the boundary column passes from warp g to warp g+1 (same
//    CTA or the next CTA): chunk j of the producer (its CH tail-lane values)
//    goes by two vector asynchronous stores into slot j of g+1's ring, whose
//    mbarrier the stores complete; consumer chunk c reads slots c+3 and
//    c+4 (the 31-row skew between neighbouring strips), and a relaxed
//    counter of released slots keeps the producer from overwriting early.
//  - Between waves the last strip's boundary column goes through global
//    memory, announced by a counter in CTA 0 (release / acquire).
// Spreading the strips over CL SMs multiplies the bandwidth that feeds the
// recurrences.  All waits are bounded.
//
// LA (two-step form): substituting the recurrence into itself once gives,
// for step t+1 of lane l with n = the upstream lane (l+1 forward, l-1
// reversed),
//     z_{t+1}(l) = K + A z_{t-1}(l) + B z_{t-1}(n) + C z_{t-1}(n'),  n' = n's upstream lane,
//     K = beta_{t+1} - cV_{t+1} beta_t(l) - cH_{t+1} beta_t(n),
//     A = cV_{t+1} cV_t(l),  B = cV_{t+1} cH_t(l) + cH_{t+1} cV_t(n),  C = cH_{t+1} cH_t(n),
// so the dependency chain advances two steps per three FMAs instead of four;
// z_t(l) itself is formed beside it, off the chain.  The head lane's
// upstream value z_t(n) is the boundary value it receives, so it takes
// n's coefficients as zero and n's beta as that value; the lane next to it
// takes its z_{t-1}(n') from the boundary as well.  Same arithmetic as the
// sequential sweep up to rounding order.
template <typename T, bool REV, int CH, bool BND, bool LA>
__global__ void __launch_bounds__(512, 1) k_dts(DtsArgs<T> A, int NST) {
    static_assert(CH == 8 || CH == 16 || CH == 32, "ring slots carry 8, 16 or 32 values");
    static_assert(!(LA && BND), "the two-step form has no boundary-vector variant");
    constexpr int DTS_RS = DtsRing<T, CH>::RS, DTS_NSL = DtsRing<T, CH>::NSL;
    constexpr int NSUB = CH / DTS_RS;   // ring slots per chunk
    constexpr int SKR = 31 / DTS_RS;    // the 31-row skew spans SKR whole slots
    static_assert(CH % DTS_RS == 0 && DTS_RS % 4 == 0, "chunks hold whole ring slots");
    typedef typename Vec2T<T>::type T2;
    typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V;
    constexpr int VEC = 16 / sizeof(T);
    typedef DtsSmem<T, CH> SM;
    if (A.skip && *A.skip) return;   // same value in every CTA of the cluster
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int WC = (blockDim.x >> 5) - 1, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int W = CL * WC;
    unsigned char *const stages = smem_raw;
    unsigned char *const rings = stages + (size_t)WC * NST * SM::stage;
    unsigned long long *const fullb = reinterpret_cast<unsigned long long *>(rings + (size_t)WC * SM::ring);
    unsigned long long *const emptyb = fullb + (size_t)WC * NST;
    unsigned long long *const rbars = emptyb + (size_t)WC * NST;
    unsigned *const relc = reinterpret_cast<unsigned *>(rbars + (size_t)WC * DTS_NSL);
    unsigned *const wave_done = relc + WC;
    volatile unsigned *const abort_flag = wave_done + 1;

    const Region R = A.R;
    const int S = R.S, D = R.D, my = R.my;
    const int qoff = REV ? D - (my + 31) : 0;   // padding diagonals come first in reversed order
    const int head = REV ? 0 : 31, tail = REV ? 31 : 0;
    const int nch = D / CH;
    const int nsl = D / DTS_RS;   // ring slots per strip

    if (threadIdx.x < WC) relc[threadIdx.x] = 0u;
    if (threadIdx.x == 0) { *wave_done = 0u; *abort_flag = 0u; }
    if (w < WC && lane == 0) {
        for (int q = 0; q < NST; q++) {
            mbar_init(fullb + w * NST + q, 1);
            mbar_init(emptyb + w * NST + q, 1);
        }
        for (int q = 0; q < DTS_NSL; q++) mbar_init(rbars + w * DTS_NSL + q, 1);
        for (int q = 0; q < DTS_NSL; q++) mbar_arrive_expect_tx(rbars + w * DTS_NSL + q, (unsigned)(DTS_RS * sizeof(T)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    cluster.sync();   // every CTA initialised before any peer writes into it

    if (w == WC) {
        // ---- copy warp: lane 0 fills the stages of every compute warp ----
        if (lane == 0) {
            int kk[16], cc[16], seq[16];
            for (int i = 0; i < WC; i++) { kk[i] = 0; cc[i] = 0; seq[i] = 0; }
            int left = 0;
            for (int i = 0; i < WC; i++) left += (rank * WC + i < S) ? 1 : 0;
            long long n = 0;
            while (left > 0) {
                bool any = false;
                for (int i = 0; i < WC; i++) {
                    const int gi = rank * WC + i;
                    const int sidx = gi + kk[i] * W;
                    if (sidx >= S) continue;
                    const int q = seq[i] % NST, use = seq[i] / NST;
                    if (use > 0 && !mbar_test_wait(emptyb + i * NST + q, (unsigned)(use - 1) & 1u)) continue;
                    const int s = REV ? sidx : S - 1 - sidx;
                    const long long sbase = R.off + (((long long)s * D) << 5);
                    const int c = cc[i];
                    const int d0 = REV ? D - (c + 1) * CH : c * CH;
                    unsigned char *st = stages + ((size_t)i * NST + q) * SM::stage;
                    mbar_arrive_expect_tx(fullb + i * NST + q, (unsigned)SM::stage);
                    bulk_g2s(st, A.pair + sbase + ((long long)d0 << 5), (unsigned)SM::stage_pairs, fullb + i * NST + q);
                    bulk_g2s(st + SM::stage_pairs, A.beta + sbase + ((long long)d0 << 5), (unsigned)SM::stage_beta,
                             fullb + i * NST + q);
                    seq[i]++;
                    if (++cc[i] == nch) {
                        cc[i] = 0;
                        kk[i]++;
                        if (gi + kk[i] * W >= S) left--;
                    }
                    any = true;
                }
                if (any) {
                    n = 0;   // counts consecutive idle polls only
                } else if (++n > BLP_SPIN_LIMIT) {   // compute warps stopped consuming
                    *abort_flag = 1u;
                    atomicExch(A.err, BLP_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __syncwarp();
        cluster.sync();
        return;
    }

    // ---- compute warps ----
    const int g = rank * WC + w;
    unsigned char *const mystage = stages + (size_t)w * NST * SM::stage;
    unsigned long long *const myfull = fullb + (size_t)w * NST;
    unsigned long long *const myempty = emptyb + (size_t)w * NST;
    unsigned long long *const myrbar = rbars + (size_t)w * DTS_NSL;
    const T *const ring_w = reinterpret_cast<const T *>(rings + (size_t)w * SM::ring);
    // successor g+1 (its ring and ring mbarriers), predecessor g-1 (its
    // released-slot counter), CTA 0's wave counter: shared::cluster addresses
    const int sg = g + 1 < W ? g + 1 : g, pg = g > 0 ? g - 1 : g;
    const unsigned succ_ring = mapa_u32(smem_u32(rings) + (unsigned)((sg % WC) * SM::ring), (unsigned)(sg / WC));
    const unsigned succ_rbar = mapa_u32(smem_u32(rbars) + (unsigned)((sg % WC) * DTS_NSL * 8), (unsigned)(sg / WC));
    const unsigned pred_rel = mapa_u32(smem_u32(relc) + (unsigned)((pg % WC) * 4), (unsigned)(pg / WC));
    const unsigned wave_cta0 = mapa_u32(smem_u32(wave_done), 0u);

    int k_in = 0, k_out = 0;   // strips consumed from g-1 / produced for g+1
    int seq = 0;               // chunks taken from the stages
    int rel_seen = 0;          // successor's released-slot count as last read (it only grows)

    for (int k = 0;; k++) {
        const int sidx = g + k * W;
        if (sidx >= S) break;
        const int s = REV ? sidx : S - 1 - sidx;
        const bool has_in = g > 0;
        const bool from_global = g == 0 && sidx > 0;
        const bool has_out = (g + 1 < W) && (sidx + 1 < S);
        const int sprev = REV ? s - 1 : s + 1;
        const long long sbase = R.off + (((long long)s * D) << 5);
        if (from_global) wait_counter(wave_done, k, abort_flag, A.err);   // g == 0 lives in CTA 0
        int waited = 0, released = 0;   // ring slots of this strip waited for / released
        T zprev = T(0);
        T *const outp = A.out + sbase + lane;
        for (int c = 0; c < nch; c++) {
            const int t0 = c * CH;
            T hz[CH];
#pragma unroll
            for (int u = 0; u < CH; u++) hz[u] = T(0);
            if (from_global) {
#pragma unroll
                for (int u = 0; u < CH; u++) {
                    const int t = t0 + u;
                    const int ktop = REV ? D - 1 - t - 31 : t;
                    const int dprev = REV ? ktop : ktop + 31;
                    if ((LA || lane == head) && ktop >= 0 && ktop < my)
                        hz[u] = __ldcg(A.out + R.off + (((long long)sprev * D + dprev) << 5) + (REV ? 31 : 0));
                }
            }
            const int q = seq % NST;
            mbar_wait(myfull + q, (unsigned)(seq / NST) & 1u, abort_flag, A.err);
            const T2 *const pp = reinterpret_cast<const T2 *>(mystage + (size_t)q * SM::stage);
            const T *const pb = reinterpret_cast<const T *>(mystage + (size_t)q * SM::stage + SM::stage_pairs);
            const bool is_head = lane == head;
            T *const op = outp + ((long long)(REV ? D - 1 - t0 : t0) << 5);
            T tz[CH];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                const int n = c * NSUB + i;   // sub-chunk of this strip: steps t0 + i*RS .. +RS-1
                if (has_in) {
                    const int upto = min(n + SKR + 1, nsl - 1);
                    for (; waited <= upto; waited++) {
                        const int P = k_in * nsl + waited;
                        mbar_wait_cluster(myrbar + P % DTS_NSL, (unsigned)(P / DTS_NSL) & 1u, abort_flag, A.err);
                    }
                    // row t0+u-qoff left the producer at its step t0+u+31: slot
                    // (t0+u+31)/RS, value (t0+u+31) % RS, i.e. for u = i*RS + j the
                    // last value of slot n+SKR (j = 0) or value j-1 of slot n+SKR+1
                    const int Pa = k_in * nsl + n + SKR, Pb = Pa + 1;
                    const T *sa = ring_w + (Pa % DTS_NSL) * DTS_RS, *sb = ring_w + (Pb % DTS_NSL) * DTS_RS;
                    T sbv[DTS_RS];
#pragma unroll
                    for (int e = 0; e < DTS_RS; e += VEC)   // slots are 16-byte aligned: vector reads
                        *reinterpret_cast<V *>(sbv + e) = *reinterpret_cast<const V *>(sb + e);
#pragma unroll
                    for (int j = 0; j < DTS_RS; j++) {
                        const int row = t0 + i * DTS_RS + j - qoff;
                        const T v = j == 0 ? sa[DTS_RS - 1] : sbv[j - 1];
                        hz[i * DTS_RS + j] = (row >= 0 && row < my) ? v : T(0);
                    }
                }
                // The successor's ring slot for this sub-chunk (P): free once the
                // successor has released P - DTS_NSL + 1 slots (its counter is read only
                // when the last value seen does not show that).  In the one-step form the tail
                // lane stores each 16 bytes of the slot as soon as the steps have
                // produced them: the stores issue in the shadow of the recurrence's
                // latency and the slot completes one store after its last step
                // (FP64 sweeps 6.5% faster, measured).
                constexpr int E = 16 / (int)sizeof(T);   // values per 16-byte piece
                const bool st_on = has_out && lane == tail;
                unsigned slot = 0u, sbar = 0u;
                if (!LA && has_out) {
                    const int P = k_out * nsl + n;   // slot sequence number in the successor's ring
                    if (P - DTS_NSL + 1 > rel_seen) rel_seen = wait_counter(relc + w, P - DTS_NSL + 1, abort_flag, A.err);
                    slot = succ_ring + (unsigned)((P % DTS_NSL) * DTS_RS * sizeof(T));
                    sbar = succ_rbar + (unsigned)((P % DTS_NSL) * 8);
                }
                if constexpr (LA) {
                    const bool next_head = lane == (REV ? 1 : 30);
                    const int nl = REV ? max(lane - 1, 0) : min(lane + 1, 31);   // upstream lane (clamped)
#pragma unroll
                    for (int u = i * DTS_RS; u < i * DTS_RS + DTS_RS; u += 2) {
                        const int ui0 = REV ? CH - 1 - u : u, ui1 = REV ? CH - 2 - u : u + 1;
                        const T2 c0 = pp[ui0 * 32 + lane], c1 = pp[ui1 * 32 + lane];
                        const T b0 = pb[ui0 * 32 + lane], b1 = pb[ui1 * 32 + lane];
                        T2 n0 = pp[ui0 * 32 + nl];
                        T nb0 = pb[ui0 * 32 + nl];
                        if (is_head) { n0.x = T(0); n0.y = T(0); nb0 = hz[u + 1]; }
                        const T K = b1 - c1.y * b0 - c1.x * nb0;
                        const T Ac = c1.y * c0.y, Bc = c1.y * c0.x + c1.x * n0.y, Cc = c1.x * n0.x;
                        T Z1 = REV ? __shfl_up_sync(FULL, zprev, 1) : __shfl_down_sync(FULL, zprev, 1);
                        T Z2 = REV ? __shfl_up_sync(FULL, zprev, 2) : __shfl_down_sync(FULL, zprev, 2);
                        Z1 = is_head ? hz[u] : Z1;
                        Z2 = is_head ? T(0) : (next_head ? hz[u] : Z2);
                        T z1 = K + Ac * zprev;
                        z1 = z1 + Bc * Z1;
                        z1 = z1 + Cc * Z2;
                        T z0 = b0 - c0.y * zprev;
                        z0 = z0 - c0.x * Z1;
                        op[REV ? -(u << 5) : (u << 5)] = z0;
                        op[REV ? -((u + 1) << 5) : ((u + 1) << 5)] = z1;
                        tz[u] = z0;
                        tz[u + 1] = z1;
                        zprev = z1;
                    }
                } else {
#pragma unroll
                    for (int u = i * DTS_RS; u < i * DTS_RS + DTS_RS; u++) {
                        const int ui = REV ? CH - 1 - u : u;
                        const T2 cpair = pp[ui * 32 + lane];
                        const T beta = pb[ui * 32 + lane];
                        T zH = REV ? __shfl_up_sync(FULL, zprev, 1) : __shfl_down_sync(FULL, zprev, 1);
                        zH = is_head ? hz[u] : zH;
                        T zV = zprev;
                        if (BND) {   // reversed interior sweep: west / south neighbours in the X / Y blocks
                            const int ktop = (REV ? D - 1 - (t0 + u) : t0 + u) - 31 + lane;
                            const int a = s * 32 + lane, b = my - 1 - ktop;
                            if (ktop >= 0 && ktop < my && a < R.mx) {
                                if (a == 0) zH = A.bnd[A.lay.addr(R.i0 - 1, R.j0 + b)];
                                if (b == 0) zV = A.bnd[A.lay.addr(R.i0 + a, R.j0 - 1)];
                            }
                        }
                        T z = beta - cpair.y * zV;
                        z = z - cpair.x * zH;
                        op[REV ? -(u << 5) : (u << 5)] = z;
                        tz[u] = z;
                        zprev = z;
                        if ((u + 1 - i * DTS_RS) % E == 0)
                            st_async_16(st_on, slot + (unsigned)((u + 1 - E - i * DTS_RS) * sizeof(T)), tz + u + 1 - E, sbar);
                    }
                }
                // The two-step form checks and stores its slot after the steps: issued
                // inside its short steps the stores made the FP32 sweep 50% slower, and
                // the check before them 2% slower (measured).
                if (LA && has_out) {
                    const int P = k_out * nsl + n;
                    if (P - DTS_NSL + 1 > rel_seen) rel_seen = wait_counter(relc + w, P - DTS_NSL + 1, abort_flag, A.err);
                    if (st_on)
                        st_async_rs<DTS_RS>(succ_ring + (unsigned)((P % DTS_NSL) * DTS_RS * sizeof(T)), tz + i * DTS_RS,
                                            succ_rbar + (unsigned)((P % DTS_NSL) * 8));
                }
                // Slots no later sub-chunk reads are re-armed for their next use and
                // released every eighth sub-chunk and at the strip's end (one warp-wide
                // branch and two warp barriers per eight slots).  The count the
                // predecessor sees trails the true count by at most seven slots, while
                // the producer needs it only DTS_NSL - 1 slots ahead of the slots this
                // warp still waits for (n + SKR + 1); a slot is re-armed at least
                // DTS_NSL - 8 slots before this warp waits on its next phase.
                if ((n & 7) == 7 || n == nsl - 1) {
                    __syncwarp();   // every lane has read the ring slots released here
                    if (has_in && lane == head && !*abort_flag) {
                        const int rel = n == nsl - 1 ? nsl : min(n + SKR + 1, nsl);
                        for (; released < rel; released++) {
                            const int P = k_in * nsl + released;
                            mbar_arrive_expect_tx(myrbar + P % DTS_NSL, (unsigned)(DTS_RS * sizeof(T)));
                        }
                        st_relaxed_cluster(pred_rel, (unsigned)(k_in * nsl + released));
                    }
                    __syncwarp();
                }
            }
            if (lane == 0) mbar_arrive(myempty + q);   // stage read: the copy warp may refill it
            seq++;
        }
        if (has_in) k_in++;
        if (has_out) k_out++;
        // the next wave's first warp reads this strip's boundary column from global memory
        if (g == W - 1 && sidx + 1 < S && lane == tail) st_release_cluster(wave_cta0, (unsigned)(k + 1));
    }
    __syncwarp();
    cluster.sync();
}

// Self-check of the bounded waits: one warp waits, with the kernels' own
// helpers and a short iteration limit, for a counter and an mbarrier phase
// that nothing completes.  Each wait must give up, record BLP_ERR_TIMEOUT
// and return; err[0] / err[1] receive the two outcomes.
__global__ void k_wait_probe(int *err, long long limit) {
    __shared__ unsigned ctr;
    __shared__ unsigned abort_flag;
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        ctr = 0u;
        abort_flag = 0u;
        mbar_init(&bar, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();
    wait_counter(&ctr, 1, &abort_flag, err, limit);
    __syncwarp();
    if (threadIdx.x == 0) abort_flag = 0u;
    __syncwarp();
    mbar_wait_cluster(&bar, 0u, &abort_flag, err + 1, limit);
}

extern "C" int blp_check_wait_timeout(blp_handle *h) {
    if (!h) return BLP_ERR_ARG;
    int res[2] = {0, 0};
    CUDA_TRY(cudaMemsetAsync(h->err, 0, 2 * sizeof(int), h->stream));
    k_wait_probe<<<1, 32, 0, h->stream>>>(h->err, 2000);
    LAUNCH_CHECK(h);
    CUDA_TRY(cudaMemcpyAsync(res, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemsetAsync(h->err, 0, 2 * sizeof(int), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return (res[0] == BLP_ERR_TIMEOUT && res[1] == BLP_ERR_TIMEOUT) ? BLP_ERR_TIMEOUT : BLP_OK;
}

// Cluster shape for a block of S strips: CL <= max_cluster CTAs (one per
// SM: the dynamic shared memory is padded so that two CTAs cannot share an
// SM) of WC <= 15 compute warps, and as many bulk-copy stages as fit.
struct DtsShape { int CL, WC, NST; size_t smem; };
template <typename T, int CH>
static DtsShape dts_shape(int S, int max_cluster) {
    typedef DtsSmem<T, CH> SM;
    const size_t cap = 225 * 1024;
    DtsShape sh;
    sh.CL = std::max(1, std::min(max_cluster, S));
    sh.WC = std::min(15, (S + sh.CL - 1) / sh.CL);
    sh.CL = std::min(sh.CL, (S + sh.WC - 1) / sh.WC);
    sh.NST = 16;
    while (sh.NST > 2 && SM::bytes(sh.WC, sh.NST) > cap) sh.NST--;
    sh.smem = SM::bytes(sh.WC, sh.NST);
    if (sh.CL > 1) sh.smem = std::max(sh.smem, (size_t)120 * 1024);
    return sh;
}

template <typename T, int CH>
static bool dts_fits(int S, int max_cluster, int min_stages) {
    const DtsShape sh = dts_shape<T, CH>(S, max_cluster);
    return sh.NST >= min_stages && DtsSmem<T, CH>::bytes(sh.WC, sh.NST) <= 225 * 1024;
}

template <typename K>
static bool dts_attrs(K kern) {
    // clusters above 8 CTAs are non-portable and must be allowed per kernel
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// the attributes of every form of one (precision, direction, chunk), set
// once per process (also before a capture: attributes are not set inside one)
template <typename T, bool REV, int CH>
static bool dts_attrs_once() {
    constexpr bool HAS_LA = CH >= 16;   // the 8-row fallback keeps the one-step form
    static std::atomic<bool> attr_set{false};
    if (!attr_set) {
        if (!dts_attrs(k_dts<T, REV, CH, false, false>) || !dts_attrs(k_dts<T, REV, CH, true, false>) ||
            (HAS_LA && !dts_attrs(k_dts<T, REV, CH, false, HAS_LA>)))
            return false;
        attr_set = true;
    }
    return true;
}
template <typename T>
static bool dts_attrs_all() {
    return dts_attrs_once<T, false, 8>() && dts_attrs_once<T, false, 16>() && dts_attrs_once<T, false, 32>() &&
           dts_attrs_once<T, true, 8>() && dts_attrs_once<T, true, 16>() && dts_attrs_once<T, true, 32>();
}

template <typename T, bool REV, int CH>
static int launch_dts_ch(blp_handle *h, const DtsArgs<T> &a, int cls, bool la) {
    constexpr bool HAS_LA = CH >= 16;   // the 8-row fallback keeps the one-step form
    if (!dts_attrs_once<T, REV, CH>()) return BLP_ERR_CUDA;
    const DtsShape sh = dts_shape<T, CH>(a.R.S, h->dts_max_cluster);
    if (DtsSmem<T, CH>::bytes(sh.WC, sh.NST) > 225 * 1024) return BLP_ERR_ARG;
    // algorithmic words per node: beta, two couplings, out; the chain has one
    // step per anti-diagonal, mx + my - 1 of them
    ProfScope ps(h, cls, (double)a.R.mx * a.R.my * sizeof(T) * 4, (double)(a.R.mx + a.R.my - 1));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sh.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(sh.CL);
    cfg.blockDim = dim3((sh.WC + 1) * 32);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = a.bnd             ? cudaLaunchKernelEx(&cfg, k_dts<T, REV, CH, true, false>, a, sh.NST)
                    : (HAS_LA && la) ? cudaLaunchKernelEx(&cfg, k_dts<T, REV, CH, false, HAS_LA>, a, sh.NST)
                                     : cudaLaunchKernelEx(&cfg, k_dts<T, REV, CH, false, false>, a, sh.NST);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BLP_ERR_CUDA;
    }
    LAUNCH_CHECK(h);
    return BLP_OK;
}

template <typename T, bool REV>
static int launch_dts(blp_handle *h, const DtsArgs<T> &a, int cls) {
    // default: 32 rows in FP32 (the per-chunk hand-off dominates a 38-cycle
    // step), 16 in FP64 (a 220-cycle step dominates; shorter lag)
    // shorter chunks where the cluster shape's stages would not fit (many
    // warps per CTA on the largest blocks); the 32-row chunk only with at
    // least 4 stages of prefetch
    int ch = h->dts_chunk ? h->dts_chunk : (sizeof(T) == 4 ? 32 : 16);
    if (ch == 32 && !dts_fits<T, 32>(a.R.S, h->dts_max_cluster, 4)) ch = 16;
    if (ch == 16 && !dts_fits<T, 16>(a.R.S, h->dts_max_cluster, 2)) ch = 8;
    const bool la = sizeof(T) == 4 ? h->dts_two_step32 : h->dts_two_step64;
    if (ch == 8) return launch_dts_ch<T, REV, 8>(h, a, cls, la);
    if (ch == 32) return launch_dts_ch<T, REV, 32>(h, a, cls, la);
    return launch_dts_ch<T, REV, 16>(h, a, cls, la);
}

