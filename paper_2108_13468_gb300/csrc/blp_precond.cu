// blp_precond.cu -- the boundary-layer preconditioner of Sec. 3.1,
// eq. (2D blocks), applied to the row-normalised system, and its transpose.
//
//   interior block I : M_II, downstream Gauss-Seidel    -> wavefront kernel
//   edge blocks Y, X : M_YY / M_XX, ordered line solves -> line-chain kernel
//   corner block C   : M_CC, multigrid iteration (Sec. 3.2) -> wavefront
//                      smoother + fused restriction / prolongation kernels
#include "blp_common.cuh"
#include <algorithm>

#define FULL 0xffffffffu

// ---------------------------------------------------------------------------
// Wavefront kernel: downstream triangular solve on a SKEW block
//     z(a,b) = beta(a,b) - cV(a,b) zV - cH(a,b) zH
// forward (REV = false): zH = z(a+1,b) (east), zV = z(a,b+1) (north), the
//   sweep starts at the top-right node (Sec. 3.1 M_II; Sec. 3.2 smoother);
// reversed (REV = true): zH = z(a-1,b), zV = z(a,b-1), starting bottom-left
//   (the transposed sweeps of the adjoint).
// GS = true makes it one Gauss-Seidel sweep of the full 5-point operator:
//   beta = b - oH * e_old(other horizontal neighbour) - oV * e_old(other
//   vertical neighbour), which equals the sequential sweep exactly because
//   those neighbours come later in the sweep order.
// One CTA, warp w owns strips in processing order w, w+W, ...; lane l owns
// column 32s+l and handles diagonal d at step t (d = t forward, D-1-t
// reversed).  The lane next to the previous strip ("head") takes that
// strip's boundary column from a shared-memory ring filled by the warp that
// processed it; all waits are bounded and report BLP_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
template <typename T>
struct DtsArgs {
    Region R;
    const T *rhs;      // beta (plain) or b (Gauss-Seidel)
    const T *eold;     // Gauss-Seidel: previous iterate
    T *out;
    const T *cH, *cV;  // chain couplings
    const T *oH, *oV;  // Gauss-Seidel couplings to not-yet-updated neighbours
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

template <typename T, bool GS, bool REV>
__global__ void __launch_bounds__(1024) k_dts(DtsArgs<T> A) {
    if (A.skip && *A.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *ring = reinterpret_cast<T *>(smem_raw);
    volatile int *prod = reinterpret_cast<volatile int *>(ring + (size_t)W * BLP_RING);
    volatile int *cons = prod + W;
    volatile int *abort_flag = cons + W;
    if (threadIdx.x < W) { prod[threadIdx.x] = 0; cons[threadIdx.x] = 0; }
    if (threadIdx.x == 0) *abort_flag = 0;
    __syncthreads();

    const Region R = A.R;
    const int S = R.S, D = R.D, my = R.my, mx = R.mx;
    const int head = REV ? 0 : 31, tail = REV ? 31 : 0;
    const int wnext = (w + 1) % W;
    const int rounds = (S - w + W - 1) / W;
    int in_seq = 0, out_seq = 0, cached_prod = 0, cached_cons = 0;

    for (int k = 0; k < rounds; k++) {
        const int sidx = w + k * W;
        const int s = REV ? sidx : S - 1 - sidx;
        const bool has_in = sidx > 0, has_out = sidx + 1 < S;
        const int a = s * 32 + lane;
        const long long base = R.off + (((long long)s * D) << 5) + lane;
        T zprev = T(0);
        for (int t = 0; t < D; t++) {
            const int d = REV ? D - 1 - t : t;
            const int ktop = d - 31 + lane;
            const bool valid = (a < mx) && ktop >= 0 && ktop < my;
            const int b = my - 1 - ktop;
            const long long p = base + ((long long)d << 5);

            T zring = T(0);
            if (lane == head && has_in && t < my) {
                const int seq = in_seq + t;
                if (seq >= cached_prod) {
                    spin_wait_ge(prod + w, seq + 1, abort_flag, A.err);
                    cached_prod = prod[w];
                }
                __threadfence_block();
                zring = ring[(size_t)w * BLP_RING + (seq % BLP_RING)];
                if ((t & 15) == 15 || t == my - 1) {
                    __threadfence_block();
                    cons[w] = seq + 1;
                }
            }
            T zH = REV ? __shfl_up_sync(FULL, zprev, 1) : __shfl_down_sync(FULL, zprev, 1);
            if (lane == head) zH = zring;
            T zV = zprev;

            T z = T(0);
            if (valid) {
                if (REV && A.bnd) {
                    if (a == 0) zH = A.bnd[A.lay.addr(R.i0 - 1, R.j0 + b)];
                    if (b == 0) zV = A.bnd[A.lay.addr(R.i0 + a, R.j0 - 1)];
                }
                T beta = A.rhs[p];
                if (GS) {
                    const int ah = REV ? a + 1 : a - 1;
                    const int bv = REV ? b + 1 : b - 1;
                    if (ah >= 0 && ah < mx) beta -= A.oH[p] * A.eold[R.addr(ah, b)];
                    if (bv >= 0 && bv < my) beta -= A.oV[p] * A.eold[R.addr(a, bv)];
                }
                z = beta - A.cV[p] * zV;
                z = z - A.cH[p] * zH;
            }
            A.out[p] = z;

            if (lane == tail && has_out) {
                const int q = t - 31;
                if (q >= 0 && q < my) {
                    const int seq = out_seq + q;
                    if (seq - cached_cons >= BLP_RING) {
                        spin_wait_ge(cons + wnext, seq - BLP_RING + 1, abort_flag, A.err);
                        cached_cons = cons[wnext];
                    }
                    ring[(size_t)wnext * BLP_RING + (seq % BLP_RING)] = z;
                    __threadfence_block();
                    prod[wnext] = seq + 1;
                }
            }
            zprev = z;
        }
        if (has_in) in_seq += my;
        if (has_out) out_seq += my;
    }
}

template <typename T, bool GS, bool REV>
static int launch_dts(blp_handle *h, const DtsArgs<T> &a) {
    int W = std::min(a.R.S, 32);
    size_t smem = (size_t)W * BLP_RING * sizeof(T) + sizeof(int) * (2 * W + 2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_dts<T, GS, REV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    k_dts<T, GS, REV><<<1, W * 32, smem, h->stream>>>(a);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

// ---------------------------------------------------------------------------
// Block-wide scan of an affine recurrence x_e = alpha_e + mu_e x_{e-1}
// (BACK = false, e ascending) or x_e = alpha_e + mu_e x_{e+1} (BACK = true),
// x = 0 outside the sequence.  Thread t owns elements [t*KPT, t*KPT+KPT).
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
    // inclusive scan over lanes in sequence order (ascending lanes forward,
    // descending lanes backward)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T Ap = BACK ? __shfl_down_sync(FULL, A, off) : __shfl_up_sync(FULL, A, off);
        T Mp = BACK ? __shfl_down_sync(FULL, M, off) : __shfl_up_sync(FULL, M, off);
        const bool ok = BACK ? (lane + off < 32) : (lane >= off);
        if (ok) { A = A + M * Ap; M = M * Mp; }
    }
    const int last = BACK ? 0 : 31;
    if (lane == last) { sh[wid] = A; sh[32 + wid] = M; }
    __syncthreads();
    // carry into this warp: compose the totals of the warps before it
    T carry = T(0);
    {
        const int src = BACK ? nw - 1 - lane : lane;   // sequence position -> warp id
        T Aw = (lane < nw) ? sh[src] : T(0);
        T Mw = (lane < nw) ? sh[32 + src] : T(1);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            T Ap = __shfl_up_sync(FULL, Aw, off);
            T Mp = __shfl_up_sync(FULL, Mw, off);
            if (lane >= off) { Aw = Aw + Mw * Ap; Mw = Mw * Mp; }
        }
        const int pos = BACK ? nw - 1 - wid : wid;     // this warp's position in sequence order
        T c = __shfl_sync(FULL, Aw, (pos + 31) & 31);
        carry = pos > 0 ? c : T(0);
    }
    __syncthreads();
    T Aprev = BACK ? __shfl_down_sync(FULL, A, 1) : __shfl_up_sync(FULL, A, 1);
    T Mprev = BACK ? __shfl_down_sync(FULL, M, 1) : __shfl_up_sync(FULL, M, 1);
    const bool first = BACK ? (lane == 31) : (lane == 0);
    T xin = first ? carry : Aprev + Mprev * carry;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int e = BACK ? KPT - 1 - q : q;
        xin = al[e] + mu[e] * xin;
        x[e] = xin;
    }
}

// ---------------------------------------------------------------------------
// Line chains (Sec. 3.1): block 0 = Y block (lines of constant x, solved
// right to left, keeping the E coupling to the line solved before and, on
// the top node, the N coupling into I), block 1 = X block (lines of constant
// y, top down, keeping the N coupling and, on the right node, the E coupling
// into I).  TRANS: the transposed block solves (Y left to right, X bottom up)
// with the couplings from the line before or, for the first line, from C.
// Both blocks run in one launch.  Each line: Thomas with the stored factors,
// both sweeps as block-wide affine scans.
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

template <typename T, int KPT, bool TRANS>
__global__ void __launch_bounds__(1024) k_line_chain(ChainArgs<T> A) {
    if (A.skip && *A.skip) return;
    __shared__ T sh[64];
    const bool isY = blockIdx.x == 0;
    const Layout &lay = A.lay;
    const int L = lay.L;
    const Region &C = lay.R[0], &X = lay.R[1], &Y = lay.R[2], &I = lay.R[3];
    const Region &B = isY ? Y : X;
    const int nlines = isY ? Y.mx : X.my;
    const int e0 = threadIdx.x * KPT;
    T zp[KPT], al[KPT], mu[KPT], y[KPT];
#pragma unroll
    for (int q = 0; q < KPT; q++) zp[q] = T(0);
    for (int li = 0; li < nlines; li++) {
        const int line = TRANS ? li : nlines - 1 - li;
        const long long base = B.off + (long long)line * L;
        // right-hand side of this line
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int e = e0 + q;
            if (e < L) {
                const long long s = base + e;
                T d = A.v[s];
                if (!TRANS) {
                    d -= (isY ? A.wE[s] : A.wN[s]) * zp[q];
                    if (e == L - 1) {
                        const long long pi = isY ? I.addr(line, 0) : I.addr(0, line);
                        d -= (isY ? A.wN[s] : A.wE[s]) * A.z[pi];
                    }
                } else {
                    T prev = zp[q];
                    if (li == 0) prev = A.z[isY ? C.addr(L - 1, e) : C.addr(e, L - 1)];
                    d -= (isY ? A.wET[s] : A.wNT[s]) * prev;
                }
                al[q] = d;
                mu[q] = A.lf[s];
            } else {
                al[q] = T(0);
                mu[q] = T(1);
            }
        }
        block_affine_scan<T, KPT, false>(al, mu, y, sh);
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int e = e0 + q;
            if (e < L) {
                const long long s = base + e;
                al[q] = A.lg[s] * y[q];
                mu[q] = A.lh[s];
            } else {
                al[q] = T(0);
                mu[q] = T(1);
            }
        }
        block_affine_scan<T, KPT, true>(al, mu, zp, sh);
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int e = e0 + q;
            if (e < L) A.z[base + e] = zp[q];
            else zp[q] = T(0);
        }
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
    if (L <= 4096) {
        int nt = ((L + 3) / 4 + 31) / 32 * 32;
        k_line_chain<T, 4, TRANS><<<2, nt, 0, h->stream>>>(a);
    } else {
        int nt = ((L + 7) / 8 + 31) / 32 * 32;
        k_line_chain<T, 8, TRANS><<<2, nt, 0, h->stream>>>(a);
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
    const T *b0;         // level-0 right-hand side
    const int *skip;

    int gs(int l, const T *b) {
        Level<T> &Lv = H->lev[l];
        DtsArgs<T> a;
        a.R = Lv.R; a.rhs = b; a.eold = Lv.e[cur[l]]; a.out = Lv.e[cur[l] ^ 1];
        if (!TRANS) { a.cH = Lv.wE; a.cV = Lv.wN; a.oH = Lv.wW; a.oV = Lv.wS; }
        else { a.cH = Lv.wET; a.cV = Lv.wNT; a.oH = Lv.wWT; a.oV = Lv.wST; }
        a.bnd = nullptr; a.lay = h->lay; a.skip = skip; a.err = h->err;
        int rc = launch_dts<T, true, TRANS>(h, a);
        cur[l] ^= 1;
        return rc;
    }
    int vcycle(int l) {
        Level<T> &Lv = H->lev[l];
        const T *b = l == 0 ? b0 : Lv.b;
        if (l == H->nlev - 1) {
            for (int s = 0; s < 4; s++) { int rc = gs(l, b); if (rc) return rc; }
            return BLP_OK;
        }
        int rc = gs(l, b);
        if (rc) return rc;
        Level<T> &Cn = H->lev[l + 1];
        k_mg_restrict<T, TRANS><<<grid_for(Cn.R.size, 256), 256, 0, h->stream>>>(Lv, b, Lv.e[cur[l]], Cn, Cn.b,
                                                                                Cn.e[cur[l + 1]], skip);
        LAUNCH_CHECK(h);
        rc = vcycle(l + 1);
        if (rc) return rc;
        k_mg_prolong<T, TRANS><<<grid_for(Lv.R.size, 256), 256, 0, h->stream>>>(Lv, Lv.e[cur[l]], Cn, Cn.e[cur[l + 1]], skip);
        LAUNCH_CHECK(h);
        return gs(l, b);
    }
};

// M_CC^{-1} b0 (or M_CC^{-T} b0) by the stationary multigrid iteration from
// e = 0; the result is left in the returned level-0 buffer.
template <typename T, bool TRANS>
static int corner_solve(blp_handle *h, const T *b0, T **result, int *cycles_out) {
    Hierarchy<T> &H = hier_of<T>(h);
    Cycler<T, TRANS> cy;
    cy.h = h; cy.H = &H; cy.b0 = b0;
    for (int l = 0; l < H.nlev; l++) cy.cur[l] = 0;
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
        k_corner_norm<T, TRANS><<<nb, 256, 0, h->stream>>>(L0, b0, L0.e[0], 0, h->partials, nullptr);
        LAUNCH_CHECK(h);
        k_corner_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 0, red2, h->p.corner_max_cycles);
        LAUNCH_CHECK(h);
        cy.skip = done;
        int batch = std::max(2, std::min(h->last_cycles > 0 ? h->last_cycles : 6, h->p.corner_max_cycles));
        int enq = 0;
        for (;;) {
            for (int c = 0; c < batch && enq < h->p.corner_max_cycles; c++, enq++) {
                int rc = cy.vcycle(0);
                if (rc) return rc;
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
        a.R = lay.R[3]; a.rhs = v; a.eold = nullptr; a.out = z;
        a.cH = c.wE; a.cV = c.wN; a.oH = nullptr; a.oV = nullptr;
        a.bnd = nullptr; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, false, false>(h, a))) return rc;
        // Y and X blocks
        if ((rc = launch_chains<T, false>(h, c, v, z, nullptr))) return rc;
        // C block
        T *b0 = H.lev[0].b;
        k_corner_rhs<T><<<grid_for(C.size, 256), 256, 0, h->stream>>>(lay, v, z, c.wE, c.wN, b0, nullptr);
        LAUNCH_CHECK(h);
        T *e = nullptr;
        if ((rc = corner_solve<T, false>(h, b0, &e, cycles))) return rc;
        CUDA_TRY(cudaMemcpyAsync(z + C.off, e, sizeof(T) * C.size, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        T *e = nullptr;
        if ((rc = corner_solve<T, true>(h, v + C.off, &e, cycles))) return rc;
        CUDA_TRY(cudaMemcpyAsync(z + C.off, e, sizeof(T) * C.size, cudaMemcpyDeviceToDevice, h->stream));
        if ((rc = launch_chains<T, true>(h, c, v, z, nullptr))) return rc;
        DtsArgs<T> a;
        a.R = lay.R[3]; a.rhs = v; a.eold = nullptr; a.out = z;
        a.cH = c.wET; a.cV = c.wNT; a.oH = nullptr; a.oV = nullptr;
        a.bnd = z; a.lay = lay; a.skip = nullptr; a.err = h->err;
        if ((rc = launch_dts<T, false, true>(h, a))) return rc;
    }
    return BLP_OK;
}

template int precond_apply<double>(blp_handle *, const double *, double *, int, int *);
template int precond_apply<float>(blp_handle *, const float *, float *, int, int *);
