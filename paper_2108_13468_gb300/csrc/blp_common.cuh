// blp_common.cuh -- internal types of the GB300 solver: the region-major
// vector layout, the handle, launch helpers.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include "../../include/blp.h"

#define BLP_MAXLEV 24
#define BLP_RING 256          // slots of the inter-warp handoff ring of the wavefront kernel
#define BLP_SPIN_LIMIT (1LL << 26)

// ---------------------------------------------------------------------------
// Region-major layout.
//
// The interior nodes are split into the four blocks of Sec. 3.1 (C, X, Y, I).
// Each block is stored contiguously, in the order best for the kernel that
// sweeps it:
//   C and I (swept by the downstream Gauss-Seidel wavefront): SKEW layout.
//     Columns are grouped into strips of 32; inside a strip, element
//     (a, b) (a = column, b = row, both from the block's lower-left corner)
//     sits on "diagonal" d = (my-1-b) + 31 - (a%32) at slot (strip*D + d)*32
//     + a%32, D = my + 31 rounded up to a multiple of 32.  A warp whose lane l owns column 32s+l and runs
//     one diagonal per step then reads 32 consecutive words per step, for
//     the top-right-first sweep and (with d run backwards) for the
//     bottom-left-first transposed sweep alike.  Slots that map outside the
//     block are padding and are kept at zero in every vector.
//   X (horizontal line solves): ROW layout, each line of constant y contiguous.
//   Y (vertical line solves):   COL layout, each line of constant x contiguous.
// Every block starts on a 32-slot boundary (so bulk copies of a strip are
// 16-byte aligned); the slots between blocks are padding as well.
// ---------------------------------------------------------------------------
enum { LAYOUT_SKEW = 0, LAYOUT_ROW = 1, LAYOUT_COL = 2 };

struct Region {
    int kind;
    int mx, my;      // columns, rows
    int i0, j0;      // global (1-based) node of local (0,0)
    long long off;   // offset of the block inside a region-major vector
    int S, D;        // SKEW: strips, diagonals per strip
    long long size;  // slots (padding included)

    __host__ __device__ long long addr(int a, int b) const {
        if (kind == LAYOUT_SKEW) {
            int s = a >> 5, l = a & 31;
            return off + ((long long)(s * D + (my - 1 - b) + 31 - l) << 5) + l;
        }
        if (kind == LAYOUT_ROW) return off + (long long)b * mx + a;
        return off + (long long)a * my + b;
    }
    // inverse map of a slot q (relative to off); returns false for padding
    __host__ __device__ bool coords(long long q, int &a, int &b) const {
        if (kind == LAYOUT_SKEW) {
            // slot counts stay far below 2^36, so the strip/diagonal split fits 32-bit arithmetic
            const int l = (int)(q & 31);
            const int t = (int)(q >> 5);
            const int s = t / D, d = t - s * D;
            a = s * 32 + l;
            int ktop = d - 31 + l;
            b = my - 1 - ktop;
            return a < mx && ktop >= 0 && ktop < my;
        }
        if (q >= (long long)mx * my) return false;
        if (kind == LAYOUT_ROW) { a = (int)(q % mx); b = (int)(q / mx); return true; }
        a = (int)(q / my); b = (int)(q % my);
        return true;
    }
};

static inline Region make_region(int kind, int mx, int my, int i0, int j0, long long off) {
    Region r;
    r.kind = kind; r.mx = mx; r.my = my; r.i0 = i0; r.j0 = j0; r.off = off;
    if (kind == LAYOUT_SKEW) {
        // D is padded to a multiple of 32 diagonals so the wavefront kernel
        // can stage whole chunks of diagonals with bulk copies
        r.S = (mx + 31) / 32; r.D = ((my + 31) + 31) / 32 * 32;
        r.size = (long long)r.S * r.D * 32;
    } else {
        r.S = 0; r.D = 0;
        r.size = ((long long)mx * my + 31) / 32 * 32;   // keep the next block 32-slot aligned
    }
    return r;
}

struct Layout {
    int N, L;            // intervals, L = N/2 (index of the transition node)
    Region R[4];         // C, X, Y, I in storage order
    long long npad;      // total slots

    // global interior node (i,j), 1 <= i,j <= N-1 -> slot
    __host__ __device__ long long addr(int i, int j) const {
        if (i <= L) {
            if (j <= L) return R[0].addr(i - 1, j - 1);
            return R[1].addr(i - 1, j - L - 1);
        }
        if (j <= L) return R[2].addr(i - L - 1, j - 1);
        return R[3].addr(i - L - 1, j - L - 1);
    }
    // slot -> global node; false for padding
    __host__ __device__ bool node(long long p, int &i, int &j) const {
        int k = 3;
        if (p < R[1].off) k = 0;
        else if (p < R[2].off) k = 1;
        else if (p < R[3].off) k = 2;
        int a, b;
        if (!R[k].coords(p - R[k].off, a, b)) return false;
        i = R[k].i0 + a;
        j = R[k].j0 + b;
        return true;
    }
};

// L: the last layer index (transition node) of the block split, N/2 unless
// the general Shishkin mesh puts another number of intervals in the layer.
static inline Layout make_layout(int N, int L = -1) {
    Layout Lt;
    if (L < 0) L = N / 2;
    Lt.N = N; Lt.L = L;
    long long off = 0;
    Lt.R[0] = make_region(LAYOUT_SKEW, L, L, 1, 1, off);            off += Lt.R[0].size;
    Lt.R[1] = make_region(LAYOUT_ROW, L, N - 1 - L, 1, L + 1, off); off += Lt.R[1].size;
    Lt.R[2] = make_region(LAYOUT_COL, N - 1 - L, L, L + 1, 1, off); off += Lt.R[2].size;
    Lt.R[3] = make_region(LAYOUT_SKEW, N - 1 - L, N - 1 - L, L + 1, L + 1, off); off += Lt.R[3].size;
    // keep every block 32-slot aligned (128/256-byte vector loads)
    Lt.npad = (off + 31) & ~31LL;
    return Lt;
}

// ---------------------------------------------------------------------------
// Coefficients of the row-normalised operator D^-1 A (unit diagonal) in the
// region-major layout, for one precision.
//   w{W,E,S,N}(i,j) = a{W,E,S,N}(i,j) / aC(i,j)     (Sec. 3 stencil)
// Transposed-direction copies used by the adjoint sweeps:
//   wET(i,j) = wE(i-1,j), wNT(i,j) = wN(i,j-1), wWT(i,j) = wW(i+1,j), wST(i,j) = wS(i,j+1)
// (the couplings of row (i,j) of (D^-1 A)^T), 0 where the neighbour is outside.
// Line factors (Thomas, Sec. 3.1 M_YY / M_XX), stored in the Y (COL) and X
// (ROW) blocks of full-length arrays:
//   forward   y_k = d_k + lf_k y_{k-1}
//   backward  z_k = lg_k y_k + lh_k z_{k+1}
// and the same for the transposed line matrices (lfT, lgT, lhT).
// ---------------------------------------------------------------------------
template <typename T> struct Pair2;
template <> struct Pair2<float> { typedef float2 type; };
template <> struct Pair2<double> { typedef double2 type; };

template <typename T>
struct Coefs {
    typename Pair2<T>::type *pF = nullptr;   // (wE, wN): chain couplings of the forward interior sweep
    typename Pair2<T>::type *pR = nullptr;   // (wET, wNT): chain couplings of the reversed sweep
    T *wW = nullptr, *wE = nullptr, *wS = nullptr, *wN = nullptr;
    T *wET = nullptr, *wNT = nullptr, *wWT = nullptr, *wST = nullptr;
    T *lf = nullptr, *lg = nullptr, *lh = nullptr;
    T *lfT = nullptr, *lgT = nullptr, *lhT = nullptr;
    // multipliers of the line-chain scans, precomputed per line and thread
    // (forward / transposed chains); null where the chain kernel does not use them
    T *cpre = nullptr, *cpreT = nullptr;
};

// One level of the corner multigrid hierarchy (Sec. 3.2): a standalone
// SKEW block (off = 0) with its own coefficient and work arrays.
template <typename T>
struct Level {
    Region R;
    typename Pair2<T>::type *pF = nullptr, *pR = nullptr;   // packed chain couplings (wE,wN) / (wET,wNT)
    T *beta = nullptr;                                      // Gauss-Seidel right-hand side work array
    T *wW = nullptr, *wE = nullptr, *wS = nullptr, *wN = nullptr;
    T *wET = nullptr, *wNT = nullptr, *wWT = nullptr, *wST = nullptr;
    T *omega = nullptr;   // hb*kb*aC: weight taking the normalised residual to FE scaling
    T *dfe = nullptr;     // hb*kb
    T *e[2] = {nullptr, nullptr};
    T *b = nullptr;
    // natural (row-major m x m) copies for the fused coarse-level kernel, 10 arrays of m*m:
    // wW, wE, wS, wN, wET, wWT, wNT, wST, omega, dfe   (levels with m <= BLP_COARSE_MAX)
    T *nat = nullptr;
};

#define BLP_COARSE_MAX 128

template <typename T>
struct Hierarchy {
    int nlev = 0;
    Level<T> lev[BLP_MAXLEV];
};

// One level of the corner cycle for one parabolic and one exponential layer
// (Sec. 3.2): x-semicoarsened, width sx (columns) by m = N/2 (rows), with a
// nine-point operator.  Natural arrays are row-major (row J-1, column I-1).
// The Gauss-Seidel sweep reads its per-node data in a SKEW order: rows in
// blocks of 32 (block kb = (m - J) / 32, lane = (m - J) % 32), and node
// (I, J) of a block at step s = (sx - I) + 2 lane, slot (kb S + s) 32 + lane,
// S = sx + 62 steps per block; slots of no node are zero.
template <typename T>
struct SemiLev {
    int sx = 0, m = 0;
    int S = 0, nb = 0;              // steps per 32-row block, blocks
    long long nskew = 0;            // skew slots
    T *A9 = nullptr;                // 9 planes of sx*m, plane (dy+1)*3 + (dx+1): entry to (I+dx, J+dy)
    T *gE = nullptr, *gN = nullptr, *gNE = nullptr, *gNW = nullptr;   // skew: chain couplings a/aC
    T *c0 = nullptr;                // skew: sweep right-hand side, (b - old-value terms) / aC
    T *PW = nullptr, *PE = nullptr; // natural: interpolation weights of the odd columns from level l+1
    T *b = nullptr, *e = nullptr;   // natural
};

template <typename T>
struct SemiHier {
    int nlev = 0;
    SemiLev<T> lev[BLP_MAXLEV];
};

struct DevState {       // device scalars of the solver (double)
    double red[8];      // reduction results
    int flags[8];       // flags[0]: corner done; flags[1]: corner cycles; flags[3]: running max of cycles;
                        // flags[4]: corner cycles run since the solve began
};

// Kernel classes for the optional event timing (blp_profile).
enum {
    KC_DTS_GS = 0,      // corner multigrid Gauss-Seidel sweeps (wavefront)
    KC_DTS_INTERIOR,    // M_II sweep (wavefront)
    KC_LINE_CHAIN,      // M_YY / M_XX line chains
    KC_MG_RESTRICT,
    KC_MG_PROLONG,
    KC_CORNER_NORM,     // corner stopping residual + finish
    KC_MATVEC,
    KC_MULTIDOT,
    KC_UPDATE,
    KC_SMALL,           // reductions, Givens, scaling, combine
    KC_LAYOUT,          // layout conversion, corner rhs, copies
    KC_GS_RHS,          // parallel right-hand side of a Gauss-Seidel sweep
    KC_MG_COARSE,       // fused coarse levels of the corner multigrid
    KC_COUNT
};

struct ProfState {
    bool on = false;
    std::vector<cudaEvent_t> ev;   // pairs
    std::vector<int> cls;          // class per pending pair
    int used = 0;
    long long count[KC_COUNT] = {0};
    double ms[KC_COUNT] = {0.0};
    double bytes[KC_COUNT] = {0.0};   // algorithmic bytes of the recorded launches
    double steps[KC_COUNT] = {0.0};   // wavefront steps on the dependency chain of the recorded launches
};

struct blp_handle {
    blp_params p;
    int N, L;
    Layout lay;
    double tau_x, tau_y;
    std::vector<double> hx, hy;     // host mesh nodes
    double *x = nullptr, *y = nullptr;  // device mesh nodes (N+1)
    double *aC = nullptr;           // diagonal of A, region layout (FP64)
    double *c1 = nullptr, *c2 = nullptr, *r = nullptr;  // fields, standard layout (FP64)
    Coefs<double> cd;
    Coefs<float> cf;
    Hierarchy<double> hd;
    Hierarchy<float> hf;
    // parabolic-layer corner cycle (mesh == BLP_MESH_PARABOLIC): semicoarsened levels
    bool semi = false;
    SemiHier<double> sd;
    SemiHier<float> sf;
    // reduction scratch
    double *partials = nullptr;     // [BLP_RED_BLOCKS * BLP_PART_STRIDE + 64]
    DevState *dev = nullptr;
    DevState *host_state = nullptr; // pinned mirror
    int *err = nullptr;             // device error word (timeouts)
    cudaStream_t stream = 0;
    long long launches = 0;
    int dts_max_cluster = 8;        // CTAs per wavefront cluster (1..16)
    bool dts_two_step32 = true;     // two-step form of the wavefront recurrence, FP32 sweeps
    bool dts_two_step64 = false;    // FP64: off (its extra DFMAs cost more than the shorter chain saves)
    double tuned_ms = -1.0;         // blp_autotune: preconditioner time of the chosen setting (-1: not tuned)
    int dts_chunk = 0;              // wavefront chunk length (8, 16, 32 diagonals; 0: by precision)
    double t_setup_ms = 0.0;
    int last_cycles = 0;
    // Krylov work space (allocated lazily)
    size_t ws_bytes = 0;
    void *ws = nullptr;
    // standard-layout staging for host pointers
    double *stage[4] = {nullptr, nullptr, nullptr, nullptr};
    ProfState prof;
    // captured preconditioner applications (see precond_apply): one graph per
    // (precision, direction, corner batch), reading gv[prec] and writing gz[prec]
    struct PrecGraph {
        int trans, prec, batch, enq;
        cudaGraphExec_t exec;
        long long nlaunch;
        int cur[BLP_MAXLEV];
        bool zero[BLP_MAXLEV];
    };
    std::vector<PrecGraph> graphs;
    void *gv[2] = {nullptr, nullptr}, *gz[2] = {nullptr, nullptr};
    bool use_graphs = true;
    bool warm[2][2] = {{false, false}, {false, false}};   // [prec][trans]: one eager application first
    cudaStream_t own_stream = nullptr;   // capturable stream used when the caller's stream is the legacy one
    // whole-solve graphs (device-driven FGMRES, one per [precision][direction]):
    // every restart cycle, iteration and corner cycle is decided on the device
    // by conditional nodes; valid while the work space stays where it was
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        const void *ws = nullptr;
        int m = 0;
        // kernels per body (restart check, restart cycle, iteration, extra
        // corner cycle), for the launch counter
        long long n_restart = 0, n_cycle = 0, n_iter = 0, n_corner = 0;
    };
    SolveGraph solve_graph[2][2];
    bool solve_graphs = false;           // device-driven FGMRES (blp_params.device_driven, BLP_SOLVE_GRAPH)
    cudaStream_t cap[4] = {nullptr, nullptr, nullptr, nullptr};   // body streams of nested captures
    cudaStream_t cap_saved[4] = {nullptr, nullptr, nullptr, nullptr};
    int cap_depth = 0;
    bool capturing = false;              // a whole-solve capture is in progress
    long long corner_body_launches = 0;  // kernels of one captured corner cycle body
};

// Stream-ordered device allocation from the library pool (handle's stream).
int blp_internal_alloc(blp_handle *h, void **p, size_t bytes);
void blp_internal_free(blp_handle *h, void *p);
// Build the semicoarsened corner hierarchy of the parabolic-layer case from
// level 0 of the full-coarsening hierarchy (setup).
int blp_internal_semi_build(blp_handle *h);
void blp_internal_semi_free(blp_handle *h);
// M_CC^-1 b0 by the semicoarsening cycle (forward only): b0 in the corner
// level's skew layout (row-normalised right-hand side), the result written to
// out (corner region of a region-major vector, padding set to zero).
template <typename T> int semi_corner_solve(blp_handle *h, const T *b0, T *out, int *cycles);
// Precompute the line-chain scan multipliers of both precisions (setup).
int blp_internal_chain_pre(blp_handle *h);
// blp_setup with the handle's work issued on `stream` from the start.
int blp_internal_setup(const blp_params *p, const double *c1, const double *c2, const double *r, cudaStream_t stream,
                       blp_handle **out);

// Event timing of one launch when profiling is on (RAII around a launch).
int blp_internal_prof_flush(blp_handle *h);
struct ProfScope {
    blp_handle *h;
    int slot = -1;
    ProfScope(blp_handle *h_, int cls, double bytes = 0.0, double steps = 0.0) : h(h_) {
        if (!h->prof.on) return;
        h->prof.bytes[cls] += bytes;
        h->prof.steps[cls] += steps;
        if (h->prof.used * 2 + 2 > (int)h->prof.ev.size()) blp_internal_prof_flush(h);
        slot = h->prof.used++;
        h->prof.cls[slot] = cls;
        cudaEventRecord(h->prof.ev[2 * slot], h->stream);
    }
    ~ProfScope() {
        if (slot >= 0) cudaEventRecord(h->prof.ev[2 * slot + 1], h->stream);
    }
};

#define BLP_RED_BLOCKS 296    // 2 x 148: partial-sum blocks of grid reductions
#define BLP_PART_STRIDE 65    // partial sums per block (restart + 1 <= 65)
#define BLP_SCALARS_OFF ((long long)BLP_RED_BLOCKS * BLP_PART_STRIDE)  // 64 scalars after the partials

#define CUDA_TRY(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            fprintf(stderr, "blp: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return BLP_ERR_CUDA;                                              \
        }                                                                     \
    } while (0)

#define LAUNCH_CHECK(h)                                                       \
    do {                                                                      \
        (h)->launches++;                                                      \
        cudaError_t e_ = cudaPeekAtLastError();                               \
        if (e_ != cudaSuccess) {                                              \
            fprintf(stderr, "blp: launch error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return BLP_ERR_CUDA;                                              \
        }                                                                     \
    } while (0)

// ---------------------------------------------------------------------------
// Conditional nodes inside a stream capture.  cap_handle creates a handle on
// the graph that h->stream is capturing (its value is reset to `defval` at
// every launch of the executable graph); cap_begin appends an IF or WHILE
// node on that handle and redirects h->stream to a body stream that captures
// the node's body graph until cap_end restores the enclosing stream.  Bodies
// nest up to four deep.
// ---------------------------------------------------------------------------
static inline int cap_handle(blp_handle *h, unsigned defval, cudaGraphConditionalHandle *out) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, nullptr, nullptr, nullptr));
    if (st != cudaStreamCaptureStatusActive || !g) return BLP_ERR_CUDA;
    CUDA_TRY(cudaGraphConditionalHandleCreate(out, g, defval, cudaGraphCondAssignDefault));
    return BLP_OK;
}

static inline int cap_begin(blp_handle *h, cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type) {
    if (h->cap_depth >= 4 || !h->cap[h->cap_depth]) return BLP_ERR_ARG;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive || !g) return BLP_ERR_CUDA;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = c;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    CUDA_TRY(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t bs = h->cap[h->cap_depth];
    CUDA_TRY(cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    h->cap_saved[h->cap_depth++] = h->stream;
    h->stream = bs;
    return BLP_OK;
}

static inline int cap_end(blp_handle *h) {
    if (h->cap_depth <= 0) return BLP_ERR_ARG;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);   // the body graph belongs to its node
    h->stream = h->cap_saved[--h->cap_depth];
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BLP_ERR_CUDA;
    }
    return BLP_OK;
}

// End every capture in progress after a failure (bodies first, then the
// outer one, whose graph is discarded) and clear the error state.
static inline void cap_abort(blp_handle *h) {
    while (h->cap_depth > 0) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(h->stream, &g);
        h->stream = h->cap_saved[--h->cap_depth];
    }
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(h->stream, &g) == cudaSuccess && g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
}

static inline int grid_for(long long n, int threads, int cap = 152 * 8) {
    long long g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Internal entry points shared between translation units.
int blp_internal_precond(blp_handle *h, const void *v, void *z, int trans, int prec, int *cycles);
int blp_internal_ensure_ws(blp_handle *h, size_t bytes);
int blp_internal_to_region(blp_handle *h, const double *std_in, double *reg_out, int scale_mode);
int blp_internal_from_region(blp_handle *h, const double *reg_in, double *std_out, int scale_mode);
template <typename T> int precond_apply(blp_handle *h, const T *v, T *z, int trans, int *cycles);
// Set the kernel attributes of a preconditioner application before a
// whole-solve capture.
template <typename T> int precond_capture_prepare(blp_handle *h);
// Device error flag of the handle's kernels (bounded waits): BLP_OK or the
// recorded status, which it clears.
int blp_internal_check_err(blp_handle *h);
// Wavefront setting for (N, precision) chosen by the autotuner in this
// process; tunes on the given problem first when none is cached yet (null
// fields: lookup only).
int blp_internal_cached_tuning(const blp_params *p, const double *c1, const double *c2, const double *r,
                               cudaStream_t s, blp_tuning *t);
