// blp_semi.cu -- corner multigrid for one parabolic and one exponential
// layer (Sec. 3.2), the case of the mesh of eq. (tau parabolic).
//
// On that mesh the corner block is an anisotropic problem (East-West
// couplings O(N^2 / (eps ln^2 N)), North-South O(N^2 / ln^2 N)), and the
// paper approximates A_CC^-1 by cycles of a semicoarsening multigrid:
//   - inside the cycle each corner row (x_i, y_j) is rescaled by hb_i kb_j
//     (finite-element scaling), and the right-hand side with it;
//   - coarse levels halve the number of columns only (coarse column I is
//     fine column 2I; every row is kept) while the width is even, at least
//     4, and half of it at least 2;
//   - interpolation is induced by the operator: the row of fine node (i, j)
//     is collapsed North-South into three column sums s (own column), w
//     (column i-1) and e (column i+1), and an odd column takes -w/s from
//     coarse column (i-1)/2 and -e/s from (i+1)/2; even columns are
//     injected.  Entries to nodes outside the block are not entries of
//     A_CC and count as zero;
//   - restriction is P^T, each coarse operator is the Galerkin product
//     P^T A P (nine points on every coarse level);
//   - relaxation is pointwise Gauss-Seidel in the downstream order (rows
//     top to bottom, right to left in a row), V(1,1), four sweeps on the
//     coarsest level;
//   - cycles run until the scaled corner residual has fallen by the
//     handle's corner_reduction (the paper takes 10^2 here).
//
// GPU form.  The levels are built on the device at setup (FP64, then
// copied to FP32).  A Gauss-Seidel sweep of a nine-point level is a
// wavefront: node (I, J) needs the new values of (I+1, J), (I-1, J+1),
// (I, J+1) and (I+1, J+1), so with q = sx - I and r = m - J the node can be
// updated at time t = q + 2 r (the NW coupling forbids the flatter q + r).
// One CTA runs the sweep; warp w owns 32-row blocks w, w + W, ...; lane l of
// block kb owns row r = 32 kb + l and updates one node per step, taking the
// new values of the row above from lane l-1 by one shuffle per step (the
// North and North-East values are the ones it received one and two steps
// earlier).  Blocks start P steps apart; the warps advance in periods of K
// steps separated by a CTA barrier, and P >= K + 63 puts the row handed
// from block kb-1 to block kb (through global memory) at least one period
// ahead of its use.  Everything a step needs that does not depend on the
// sweep itself -- the right-hand side minus the old West, South,
// South-West and South-East terms, divided by the diagonal -- is formed
// before the sweep by a parallel kernel, and the per-node data is stored in
// the order the warps read it (one coalesced load per array and step).
#include "blp_common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

#define SFULL 0xffffffffu
#define SEMI_WARPS 16
#define STRY(x) do { int rc_ = (x); if (rc_ != BLP_OK) return rc_; } while (0)

namespace {

__host__ __device__ __forceinline__ int plane(int dx, int dy) { return (dy + 1) * 3 + (dx + 1); }

// slot of natural node (I, J) (1-based) in the skew order of a level
__host__ __device__ __forceinline__ long long skew_slot(int sx, int m, int S, int I, int J) {
    const int q = sx - I, r = m - J;
    return ((long long)(r >> 5) * S + q + 2 * (r & 31)) * 32 + (r & 31);
}

// entry of level L in row (I, J) to node (I+dx, J+dy); 0 outside the block
template <typename T>
__device__ __forceinline__ T a9(const SemiLev<T> &L, int I, int J, int dx, int dy) {
    const int In = I + dx, Jn = J + dy;
    if (In < 1 || In > L.sx || Jn < 1 || Jn > L.m) return T(0);
    return L.A9[(long long)plane(dx, dy) * L.sx * L.m + (long long)(J - 1) * L.sx + (I - 1)];
}

// ---------------------------------------------------------------------------
// set-up kernels (FP64)
// ---------------------------------------------------------------------------
// Level 0: A_0 = diag(hb kb) A_CC.  The full-coarsening level 0 holds the
// corner block row-normalised (w = a / aC) and omega = hb kb aC, so the
// scaled entries are omega and omega * w.
__global__ void k_semi_level0(Level<double> C0, SemiLev<double> L) {
    const long long n = (long long)L.sx * L.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        const long long p = C0.R.addr(I - 1, J - 1);
        const double om = C0.omega[p];
        double *A = L.A9;
        for (int q = 0; q < 9; q++) A[q * n + k] = 0.0;
        A[plane(0, 0) * n + k] = om;
        A[plane(-1, 0) * n + k] = I > 1 ? om * C0.wW[p] : 0.0;
        A[plane(1, 0) * n + k] = I < L.sx ? om * C0.wE[p] : 0.0;
        A[plane(0, -1) * n + k] = J > 1 ? om * C0.wS[p] : 0.0;
        A[plane(0, 1) * n + k] = J < L.m ? om * C0.wN[p] : 0.0;
    }
}

// Operator-induced interpolation weights of the odd columns of level L.
__global__ void k_semi_weights(SemiLev<double> L) {
    const long long n = (long long)L.sx * L.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        double pw = 0.0, pe = 0.0;
        if (I & 1) {
            const double s = a9(L, I, J, 0, -1) + a9(L, I, J, 0, 0) + a9(L, I, J, 0, 1);
            const double w = a9(L, I, J, -1, -1) + a9(L, I, J, -1, 0) + a9(L, I, J, -1, 1);
            const double e = a9(L, I, J, 1, -1) + a9(L, I, J, 1, 0) + a9(L, I, J, 1, 1);
            pw = -w / s;
            pe = -e / s;
        }
        L.PW[k] = pw;
        L.PE[k] = pe;
    }
}

// the coarse columns of level C that fine node (I, J) of level F takes
// values from, with their weights; returns how many (0..2)
__device__ __forceinline__ int pcols(const SemiLev<double> &F, int sxc, int I, int J, int *Ic, double *w) {
    if (!(I & 1)) { Ic[0] = I / 2; w[0] = 1.0; return 1; }
    const long long k = (long long)(J - 1) * F.sx + (I - 1);
    int c = 0;
    if ((I - 1) / 2 >= 1) { Ic[c] = (I - 1) / 2; w[c] = F.PW[k]; c++; }
    if ((I + 1) / 2 <= sxc) { Ic[c] = (I + 1) / 2; w[c] = F.PE[k]; c++; }
    return c;
}

// Galerkin product A_C = P^T A_F P, one coarse row per thread: the fine rows
// 2Ic-1, 2Ic, 2Ic+1 of row J carry the weights P[(2Ic-1,J),Ic] (its
// East weight), 1 and P[(2Ic+1,J),Ic] (its West weight).
__global__ void k_semi_galerkin(SemiLev<double> F, SemiLev<double> C) {
    const long long nc = (long long)C.sx * C.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nc; k += (long long)gridDim.x * blockDim.x) {
        const int Ic = (int)(k % C.sx) + 1, J = (int)(k / C.sx) + 1;
        double acc[9];
        for (int q = 0; q < 9; q++) acc[q] = 0.0;
        for (int t = -1; t <= 1; t++) {
            const int I = 2 * Ic + t;
            if (I < 1 || I > F.sx) continue;
            const long long kf = (long long)(J - 1) * F.sx + (I - 1);
            const double wp = t == 0 ? 1.0 : (t < 0 ? F.PE[kf] : F.PW[kf]);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const double a = a9(F, I, J, dx, dy);
                    if (a == 0.0) continue;
                    int Iq[2];
                    double wq[2];
                    const int nq = pcols(F, C.sx, I + dx, J + dy, Iq, wq);
                    for (int u = 0; u < nq; u++) {
                        const int ddx = Iq[u] - Ic;
                        if (ddx < -1 || ddx > 1) continue;   // P spans one coarse column each side
                        acc[plane(ddx, dy)] += wp * a * wq[u];
                    }
                }
        }
        for (int q = 0; q < 9; q++) C.A9[q * nc + k] = acc[q];
    }
}

// chain couplings of the sweep, divided by the diagonal, in skew order
__global__ void k_semi_chain_coefs(SemiLev<double> L) {
    const long long n = (long long)L.sx * L.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        const long long s = skew_slot(L.sx, L.m, L.S, I, J);
        const double c = a9(L, I, J, 0, 0);
        L.gE[s] = a9(L, I, J, 1, 0) / c;
        L.gN[s] = a9(L, I, J, 0, 1) / c;
        L.gNE[s] = a9(L, I, J, 1, 1) / c;
        L.gNW[s] = a9(L, I, J, -1, 1) / c;
    }
}

__global__ void k_semi_to_float(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

// ---------------------------------------------------------------------------
// cycle kernels
// ---------------------------------------------------------------------------
// level-0 right-hand side: bs = omega b0 (the row-normalised corner right-hand
// side taken to FE scaling), natural order; e = 0
template <typename T>
__global__ void k_semi_in(Level<T> C0, const T *__restrict__ b0, SemiLev<T> L) {
    const long long n = (long long)L.sx * L.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        const long long p = C0.R.addr(I - 1, J - 1);
        L.b[k] = C0.omega[p] * b0[p];
        L.e[k] = T(0);
    }
}

// level-0 iterate into the corner region of a region-major vector
template <typename T>
__global__ void k_semi_out(Region R, const T *__restrict__ e, int sx, T *out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < R.size; q += (long long)gridDim.x * blockDim.x) {
        int a, b;
        out[q] = R.coords(q, a, b) ? e[(long long)b * sx + a] : T(0);
    }
}

// sweep right-hand side: c0 = (b - aW eW - aS eS - aSW eSW - aSE eSE) / aC
// with the iterate before the sweep (zero: the iterate is 0)
template <typename T>
__global__ void k_semi_gsrhs(SemiLev<T> L, int zero, const int *skip) {
    if (skip && *skip) return;
    const long long n = (long long)L.sx * L.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        T c = L.b[k];
        if (!zero) {
            if (I > 1) c -= a9(L, I, J, -1, 0) * L.e[k - 1];
            if (J > 1) {
                const T *er = L.e + (k - L.sx);
                c -= a9(L, I, J, 0, -1) * er[0];
                if (I > 1) c -= a9(L, I, J, -1, -1) * er[-1];
                if (I < L.sx) c -= a9(L, I, J, 1, -1) * er[1];
            }
        }
        L.c0[skew_slot(L.sx, L.m, L.S, I, J)] = c / a9(L, I, J, 0, 0);
    }
}

// The downstream Gauss-Seidel sweep of one level (see the file comment).
// One CTA of W warps; K steps per period; blocks start P steps apart.
template <typename T, int K>
__global__ void __launch_bounds__(SEMI_WARPS * 32, 1) k_semi_gs(SemiLev<T> L, int P, const int *skip) {
    if (skip && *skip) return;
    const int sx = L.sx, m = L.m, S = L.S, nb = L.nb;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    const long long Tend = (long long)(nb - 1) * P + S;
    const long long nper = (Tend + K - 1) / K;
    T *e = L.e;
    int kb_cur = -1;
    T z1 = T(0), nw1 = T(0), nw2 = T(0);   // own last output; NW values received one and two steps ago
    for (long long per = 0; per < nper; per++) {
        const long long T0 = per * K;
        int kb = -1;
        {
            long long k0 = T0 / P;   // the latest block started by T0
            if (k0 > nb - 1) k0 = nb - 1;
            const long long kk = k0 - (((k0 - w) % W) + W) % W;   // this warp's latest block started by T0
            if (kk >= 0 && T0 < kk * P + S) kb = (int)kk;
        }
        if (kb >= 0) {
            const int s0 = (int)(T0 - (long long)kb * P);
            const int J = m - (kb * 32 + lane);   // this lane's row (< 1: no row)
            if (kb != kb_cur) {
                kb_cur = kb;
                z1 = T(0); nw2 = T(0); nw1 = T(0);
                if (lane == 0 && kb > 0) nw1 = e[(long long)J * sx + (sx - 1)];   // row J+1 at I = sx
            }
            T cc[K], cE[K], cN[K], cNE[K], cNW[K], up[K];
            const long long base = (long long)kb * S * 32 + lane;
#pragma unroll
            for (int t = 0; t < K; t++) {
                const int s = s0 + t;
                if (s < S) {
                    const long long slot = base + (long long)s * 32;
                    cc[t] = L.c0[slot]; cE[t] = L.gE[slot]; cN[t] = L.gN[slot];
                    cNE[t] = L.gNE[slot]; cNW[t] = L.gNW[slot];
                } else {
                    cc[t] = cE[t] = cN[t] = cNE[t] = cNW[t] = T(0);
                }
                // lane 0: the row above (J+1, last row of block kb-1) at q = s+1
                up[t] = (lane == 0 && kb > 0 && s + 1 < sx) ? e[(long long)J * sx + (sx - 2 - s)] : T(0);
            }
#pragma unroll
            for (int t = 0; t < K; t++) {
                const int s = s0 + t;
                const T got = __shfl_up_sync(SFULL, z1, 1);
                const T nw = lane == 0 ? up[t] : got;
                T z = cc[t] - cNE[t] * nw2 - cN[t] * nw1 - cNW[t] * nw - cE[t] * z1;
                const int q = s - 2 * lane;
                if (J >= 1 && q >= 0 && q < sx) e[(long long)(J - 1) * sx + (sx - 1 - q)] = z;
                else z = T(0);
                nw2 = nw1;
                nw1 = nw;
                z1 = z;
            }
        }
        __syncthreads();
    }
}

// residual of level F at node (I, J)
template <typename T>
__device__ __forceinline__ T semi_resid(const SemiLev<T> &F, int I, int J) {
    const long long k = (long long)(J - 1) * F.sx + (I - 1);
    T s = F.b[k];
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            const T a = a9(F, I, J, dx, dy);
            if (a != T(0)) s -= a * F.e[k + (long long)dy * F.sx + dx];
        }
    return s;
}

// coarse right-hand side P^T (b - A e) and a zero coarse iterate
template <typename T>
__global__ void k_semi_restrict(SemiLev<T> F, SemiLev<T> C, const int *skip) {
    if (skip && *skip) return;
    const long long nc = (long long)C.sx * C.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nc; k += (long long)gridDim.x * blockDim.x) {
        const int Ic = (int)(k % C.sx) + 1, J = (int)(k / C.sx) + 1;
        T acc = T(0);
        for (int t = -1; t <= 1; t++) {
            const int I = 2 * Ic + t;
            if (I > F.sx) continue;
            const long long kf = (long long)(J - 1) * F.sx + (I - 1);
            const T wgt = t == 0 ? T(1) : (t < 0 ? F.PE[kf] : F.PW[kf]);
            acc += wgt * semi_resid(F, I, J);
        }
        C.b[k] = acc;
        C.e[k] = T(0);
    }
}

// e_F += P e_C
template <typename T>
__global__ void k_semi_prolong(SemiLev<T> F, SemiLev<T> C, const int *skip) {
    if (skip && *skip) return;
    const long long n = (long long)F.sx * F.m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % F.sx) + 1, J = (int)(k / F.sx) + 1;
        const T *ec = C.e + (long long)(J - 1) * C.sx;
        T v;
        if (!(I & 1)) {
            v = ec[I / 2 - 1];
        } else {
            v = T(0);
            if ((I - 1) / 2 >= 1) v += F.PW[k] * ec[(I - 1) / 2 - 1];
            if ((I + 1) / 2 <= C.sx) v += F.PE[k] * ec[(I + 1) / 2 - 1];
        }
        F.e[k] += v;
    }
}

// squared 2-norm of b (mode 0) or of b - A e (mode 1) on level 0, one
// partial sum per block (FP64)
template <typename T>
__global__ void k_semi_norm(SemiLev<T> L, int mode, double *partials, const int *skip) {
    if (skip && *skip) return;
    const long long n = (long long)L.sx * L.m;
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(k % L.sx) + 1, J = (int)(k / L.sx) + 1;
        const double r = mode == 0 ? (double)L.b[k] : (double)semi_resid(L, I, J);
        acc += r * r;
    }
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(SFULL, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(SFULL, acc, off);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

// stopping test of the corner iteration on the device.
// mode 0: red[0] = ||b||^2 / reduction^2, flags[0] = (||b|| == 0), flags[1] = 0;
// mode 1: flags[1]++, flags[0] = 1 once ||r||^2 <= red[0] or the cycle cap is
// reached, or (stall2 > 0, FP32) once a cycle leaves ||r||^2 above stall2
// times the previous one's (red[2]): the rounding floor of an FP32 iterate
// can lie above the requested reduction.  flags[3] keeps the largest cycle
// count, flags[4] counts the cycles run.  use_cond: inside a captured solve,
// the conditional of the WHILE node that repeats the cycles is set to
// "not done" (an error flag also ends it).
__global__ void k_semi_finish(const double *partials, int nb, DevState *st, int mode, double red2, int maxc,
                              double stall2, cudaGraphConditionalHandle cond, int use_cond, const int *err) {
    if (mode == 1 && st->flags[0]) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += partials[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(SFULL, s, off);
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

template <typename T> SemiHier<T> &semi_of(blp_handle *h);
template <> SemiHier<double> &semi_of<double>(blp_handle *h) { return h->sd; }
template <> SemiHier<float> &semi_of<float>(blp_handle *h) { return h->sf; }
template <typename T> Hierarchy<T> &hier(blp_handle *h);
template <> Hierarchy<double> &hier<double>(blp_handle *h) { return h->hd; }
template <> Hierarchy<float> &hier<float>(blp_handle *h) { return h->hf; }

template <typename T> struct SweepK;
template <> struct SweepK<float> { static constexpr int K = 16; };
template <> struct SweepK<double> { static constexpr int K = 8; };

// block spacing of the sweep: a multiple of K, at least K + 63 (the hand-off
// between blocks lands a period before its use), and W P >= S (a warp's
// next block starts after its previous one ended)
static int sweep_spacing(int K, int S, int W) {
    int P = ((K + 63) + K - 1) / K * K;
    const int need = (S + W - 1) / W;
    if (need > P) P = (need + K - 1) / K * K;
    return P;
}

template <typename T>
struct SemiCycler {
    blp_handle *h;
    SemiHier<T> *H;
    const int *skip;

    int sweep(int l, bool zero) {
        SemiLev<T> &L = H->lev[l];
        const long long n = (long long)L.sx * L.m;
        {
            ProfScope ps(h, KC_GS_RHS, (double)n * (zero ? 2 : 7) * sizeof(T));
            k_semi_gsrhs<T><<<grid_for(n, 256), 256, 0, h->stream>>>(L, zero ? 1 : 0, skip);
            LAUNCH_CHECK(h);
        }
        constexpr int K = SweepK<T>::K;
        const int W = std::min(SEMI_WARPS, L.nb);
        const int P = sweep_spacing(K, L.S, W);
        // c0, 4 couplings read, e written; the chain runs sx + 2 m - 2 steps
        ProfScope ps(h, KC_DTS_GS, (double)n * 6 * sizeof(T), (double)(L.sx + 2 * L.m - 2));
        k_semi_gs<T, K><<<1, W * 32, 0, h->stream>>>(L, P, skip);
        LAUNCH_CHECK(h);
        return BLP_OK;
    }
    int vcycle(int l, bool zero) {
        SemiLev<T> &L = H->lev[l];
        if (l == H->nlev - 1) {
            for (int s = 0; s < 4; s++) STRY(sweep(l, zero && s == 0));
            return BLP_OK;
        }
        STRY(sweep(l, zero));
        SemiLev<T> &C = H->lev[l + 1];
        const long long n = (long long)L.sx * L.m, nc = (long long)C.sx * C.m;
        {
            ProfScope ps(h, KC_MG_RESTRICT, ((double)n * 11 + (double)nc * 2) * sizeof(T));
            k_semi_restrict<T><<<grid_for(nc, 256), 256, 0, h->stream>>>(L, C, skip);
            LAUNCH_CHECK(h);
        }
        STRY(vcycle(l + 1, true));
        {
            ProfScope ps(h, KC_MG_PROLONG, ((double)n * 4 + (double)nc) * sizeof(T));
            k_semi_prolong<T><<<grid_for(n, 256), 256, 0, h->stream>>>(L, C, skip);
            LAUNCH_CHECK(h);
        }
        return sweep(l, false);
    }
};

template <typename T>
int cycle_and_test(blp_handle *h, SemiCycler<T> &cy, bool first, cudaGraphConditionalHandle cond = 0, int use_cond = 0) {
    SemiLev<T> &L0 = cy.H->lev[0];
    STRY(cy.vcycle(0, first));
    const long long n = (long long)L0.sx * L0.m;
    const int nb = BLP_RED_BLOCKS;
    ProfScope ps(h, KC_CORNER_NORM, (double)n * 11 * sizeof(T));
    k_semi_norm<T><<<nb, 256, 0, h->stream>>>(L0, 1, h->partials, cy.skip);
    LAUNCH_CHECK(h);
    const double red2 = h->p.corner_reduction * h->p.corner_reduction;
    k_semi_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 1, red2, h->p.corner_max_cycles,
                                           sizeof(T) == 4 ? 0.25 : 0.0, cond, use_cond, h->err);
    LAUNCH_CHECK(h);
    return BLP_OK;
}

template <typename T>
void free_semi(blp_handle *h, SemiHier<T> &H) {
    for (int l = 0; l < H.nlev; l++) {
        SemiLev<T> &L = H.lev[l];
        T *ps[] = {L.A9, L.gE, L.gN, L.gNE, L.gNW, L.c0, L.PW, L.PE, L.b, L.e};
        for (T *p : ps) blp_internal_free(h, p);
        L = SemiLev<T>();
    }
    H.nlev = 0;
}

template <typename T>
int alloc_level(blp_handle *h, SemiLev<T> &L, int sx, int m, bool weights) {
    L.sx = sx;
    L.m = m;
    L.nb = (m + 31) / 32;
    L.S = sx + 62;
    L.nskew = (long long)L.nb * L.S * 32;
    const long long n = (long long)sx * m;
    struct { T **p; long long cnt; } want[] = {
        {&L.A9, 9 * n}, {&L.gE, L.nskew}, {&L.gN, L.nskew}, {&L.gNE, L.nskew}, {&L.gNW, L.nskew},
        {&L.c0, L.nskew}, {&L.PW, weights ? n : 0}, {&L.PE, weights ? n : 0}, {&L.b, n}, {&L.e, n}};
    for (auto &x : want) {
        if (x.cnt == 0) continue;
        void *q = nullptr;
        STRY(blp_internal_alloc(h, &q, sizeof(T) * (size_t)x.cnt));
        *x.p = static_cast<T *>(q);
        CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(T) * (size_t)x.cnt, h->stream));
    }
    return BLP_OK;
}

}  // namespace

int blp_internal_semi_build(blp_handle *h) {
    const int m = h->L;
    std::vector<int> sxs;
    int sx = m;
    for (;;) {
        sxs.push_back(sx);
        if ((sx & 1) || sx / 2 < 2 || sx < 4 || (int)sxs.size() >= BLP_MAXLEV) break;
        sx /= 2;
    }
    const int nlev = (int)sxs.size();
    h->sd.nlev = h->sf.nlev = nlev;
    for (int l = 0; l < nlev; l++) {
        STRY(alloc_level(h, h->sd.lev[l], sxs[l], m, l < nlev - 1));
        STRY(alloc_level(h, h->sf.lev[l], sxs[l], m, l < nlev - 1));
    }
    SemiLev<double> *D = h->sd.lev;
    const long long n0 = (long long)m * m;
    k_semi_level0<<<grid_for(n0, 256), 256, 0, h->stream>>>(h->hd.lev[0], D[0]);
    LAUNCH_CHECK(h);
    for (int l = 0; l + 1 < nlev; l++) {
        const long long n = (long long)D[l].sx * m, nc = (long long)D[l + 1].sx * m;
        k_semi_weights<<<grid_for(n, 256), 256, 0, h->stream>>>(D[l]);
        LAUNCH_CHECK(h);
        k_semi_galerkin<<<grid_for(nc, 256), 256, 0, h->stream>>>(D[l], D[l + 1]);
        LAUNCH_CHECK(h);
    }
    for (int l = 0; l < nlev; l++) {
        SemiLev<double> &L = D[l];
        SemiLev<float> &F = h->sf.lev[l];
        const long long n = (long long)L.sx * m;
        k_semi_chain_coefs<<<grid_for(n, 256), 256, 0, h->stream>>>(L);
        LAUNCH_CHECK(h);
        struct { const double *a; float *b; long long cnt; } cp[] = {
            {L.A9, F.A9, 9 * n}, {L.gE, F.gE, L.nskew}, {L.gN, F.gN, L.nskew}, {L.gNE, F.gNE, L.nskew},
            {L.gNW, F.gNW, L.nskew}, {L.PW, F.PW, L.PW ? n : 0}, {L.PE, F.PE, L.PE ? n : 0}};
        for (auto &c : cp) {
            if (!c.cnt) continue;
            k_semi_to_float<<<grid_for(c.cnt, 256), 256, 0, h->stream>>>(c.a, c.b, c.cnt);
            LAUNCH_CHECK(h);
        }
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->semi = true;
    return BLP_OK;
}

void blp_internal_semi_free(blp_handle *h) {
    free_semi(h, h->sd);
    free_semi(h, h->sf);
    h->semi = false;
}

template <typename T>
int semi_corner_solve(blp_handle *h, const T *b0, T *out, int *cycles_out) {
    SemiHier<T> &H = semi_of<T>(h);
    Level<T> &C0 = hier<T>(h).lev[0];
    SemiLev<T> &L0 = H.lev[0];
    const long long n0 = (long long)L0.sx * L0.m;
    {
        ProfScope ps(h, KC_LAYOUT);
        k_semi_in<T><<<grid_for(n0, 256), 256, 0, h->stream>>>(C0, b0, L0);
        LAUNCH_CHECK(h);
    }
    SemiCycler<T> cy;
    cy.h = h;
    cy.H = &H;
    cy.skip = nullptr;
    const int fixed = h->p.corner_fixed_cycles;
    int cycles = 0;
    if (fixed > 0) {
        for (int c = 0; c < fixed; c++) STRY(cy.vcycle(0, c == 0));
        cycles = fixed;
    } else {
        const int nb = BLP_RED_BLOCKS;
        const double red2 = h->p.corner_reduction * h->p.corner_reduction;
        {
            ProfScope ps(h, KC_CORNER_NORM, (double)n0 * sizeof(T));
            k_semi_norm<T><<<nb, 256, 0, h->stream>>>(L0, 0, h->partials, nullptr);
            LAUNCH_CHECK(h);
            k_semi_finish<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dev, 0, red2, h->p.corner_max_cycles, 0.0,
                                                   0, 0, nullptr);
            LAUNCH_CHECK(h);
        }
        // a batch of cycles (the count the last application needed) with the
        // stopping test on the device, then more while the test fails
        cy.skip = h->dev->flags;
        if (h->capturing) {
            // captured solve: the first cycle, then a WHILE node repeating one
            // more cycle while the stopping test fails (the cycle is in place)
            cudaGraphConditionalHandle cond;
            STRY(cap_handle(h, 0, &cond));
            STRY(cycle_and_test<T>(h, cy, true, cond, 1));
            STRY(cap_begin(h, cond, cudaGraphCondTypeWhile));
            const long long l0 = h->launches;
            const int rc = cycle_and_test<T>(h, cy, false, cond, 1);
            h->corner_body_launches = h->launches - l0;
            const int rc2 = cap_end(h);
            if (rc) return rc;
            if (rc2) return rc2;
            cycles = -1;
        } else {
            int enq = 0;
            const int batch = std::max(1, std::min(h->last_cycles > 0 ? h->last_cycles : 3, h->p.corner_max_cycles));
            for (; enq < batch; enq++) STRY(cycle_and_test<T>(h, cy, enq == 0));
            for (;;) {
                CUDA_TRY(cudaMemcpyAsync(h->host_state, h->dev, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
                CUDA_TRY(cudaStreamSynchronize(h->stream));
                if (h->host_state->flags[0] || enq >= h->p.corner_max_cycles) break;
                STRY(cycle_and_test<T>(h, cy, false));
                enq++;
            }
            cycles = h->host_state->flags[1];
            h->last_cycles = cycles;
        }
    }
    {
        ProfScope ps(h, KC_LAYOUT);
        k_semi_out<T><<<grid_for(C0.R.size, 256), 256, 0, h->stream>>>(C0.R, L0.e, L0.sx, out);
        LAUNCH_CHECK(h);
    }
    if (cycles_out) *cycles_out = cycles;
    return BLP_OK;
}

template int semi_corner_solve<double>(blp_handle *, const double *, double *, int *);
template int semi_corner_solve<float>(blp_handle *, const float *, float *, int *);
