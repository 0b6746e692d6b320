/*
 * blp_oracle.c -- plain, slow, FP64 CPU oracle for the boundary-layer
 * preconditioned solve of MacLachlan, Madden & Nhan, "A Boundary-Layer
 * Preconditioner for Singularly Perturbed Convection Diffusion"
 * (arXiv 2108.13468).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path; every routine below is written from the paper's
 * definitions in their plain sequential order, single threaded, in double
 * precision, with no blocking or fusion.
 *
 * Indexing: interior nodes (i,j), 1 <= i,j <= N-1, are stored x-fastest,
 * k = (j-1)*(N-1) + (i-1).  Mesh arrays x[0..N], y[0..N] include the
 * boundary nodes.
 *
 * Parity status of each routine (what pins it) is listed in the tests; the
 * corner multigrid coarse-grid geometry (which the paper leaves open) follows
 * the reading documented with orc_prec_create below.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_MEM 2
#define ORC_ERR_NOCONV 3
#define ORC_ERR_BREAKDOWN 4

static size_t ix(int N, int i, int j) { return (size_t)(j - 1) * (size_t)(N - 1) + (size_t)(i - 1); }

/* ------------------------------------------------------------------------
 * S0. Shishkin mesh.  Sec. 2.2, eq. (tau 1D), and Sec. 3, eq. (tau
 * exponential): tau = min(1/2, sigma*eps*ln(N)/beta); N/2 equal intervals on
 * [0,tau] and N/2 on [tau,1].  Node rule: x_i = (i/(N/2))*tau for i <= N/2,
 * x_i = tau + ((i-N/2)/(N/2))*(1-tau) above, x_N = 1 exactly.
 * Sec. 3, eq. (tau parabolic) replaces sigma*eps/beta by sigma*sqrt(eps) for a
 * parabolic layer (kind 1, beta ignored).
 *
 * kind 2: graded layer mesh.  The Remark after Theorem (big bound) notes that
 * the theory holds for graded layer meshes as well as for piecewise-uniform
 * ones; the graded mesh taken here is the Bakhvalov-Shishkin mesh (Linss,
 * J. Comput. Appl. Math. 110, 1999).  It keeps the Shishkin transition point
 * tau and the N/2 + N/2 split, and places the layer nodes so that the layer
 * function exp(-beta x / (sigma eps)) falls linearly in i:
 *     x_i = -(sigma eps / beta) ln(1 - 2 (1 - 1/N) i / N),  0 <= i <= N/2,
 * which reaches tau = sigma eps ln(N) / beta at i = N/2; uniform on [tau,1].
 * When tau is capped at 1/2 the mesh is uniform, as the Shishkin mesh is.
 * Returns tau.
 * ---------------------------------------------------------------------- */
double orc_mesh(int N, double eps, double sigma, double beta, int kind, double *x)
{
    double lnN = log((double)N);
    double tau = kind == 1 ? sigma * sqrt(eps) * lnN : sigma * eps * lnN / beta;
    int capped = tau >= 0.5;
    if (capped) tau = 0.5;
    int m = N / 2;
    for (int i = 0; i <= m; i++) {
        if (kind == 2 && !capped)
            x[i] = -(sigma * eps / beta) * log(1.0 - 2.0 * (1.0 - 1.0 / (double)N) * (double)i / (double)N);
        else
            x[i] = ((double)i / (double)m) * tau;
    }
    for (int i = m + 1; i <= N; i++) x[i] = tau + ((double)(i - m) / (double)m) * (1.0 - tau);
    x[0] = 0.0;
    x[m] = tau;
    x[N] = 1.0;
    return tau;
}

/* ------------------------------------------------------------------------
 * General Shishkin mesh (the Remark on general Shishkin meshes, Sec. 2.2):
 * a share q = NL / N of the intervals in the layer, tau = min(q,
 * sigma*eps*ln(N)/beta), NL equal intervals on [0,tau] and N - NL on
 * [tau,1]: x_i = (i/NL)*tau for i <= NL, x_i = tau + ((i-NL)/(N-NL))*(1-tau)
 * above, x_N = 1.  NL = N/2 is orc_mesh kind 0.  Returns tau.
 * ---------------------------------------------------------------------- */
double orc_mesh_q(int N, int NL, double eps, double sigma, double beta, double *x)
{
    double q = (double)NL / (double)N;
    double tau = sigma * eps * log((double)N) / beta;
    if (tau > q) tau = q;
    for (int i = 0; i <= NL; i++) x[i] = ((double)i / (double)NL) * tau;
    for (int i = NL + 1; i <= N; i++) x[i] = tau + ((double)(i - NL) / (double)(N - NL)) * (1.0 - tau);
    x[0] = 0.0;
    x[NL] = tau;
    x[N] = 1.0;
    return tau;
}

/* ------------------------------------------------------------------------
 * S1. Upwind 5-point stencil on a tensor grid (Sec. 3, the stencil display
 * after Fig. 4; 1D analogue eq. (stencil_1d)).  For an mx-by-my block of
 * nodes with coordinates xs[0..mx+1], ys[0..my+1] (index 0 and mx+1 / my+1
 * are the neighbouring nodes outside the block, treated as Dirichlet 0):
 *   W = -eps/(hb_i h_i)
 *   E = -eps/(hb_i h_{i+1}) - c1/h_{i+1}
 *   S = -eps/(kb_j k_j)
 *   N = -eps/(kb_j k_{j+1}) - c2/k_{j+1}
 *   C = eps/hb_i (1/h_i + 1/h_{i+1}) + eps/kb_j (1/k_j + 1/k_{j+1})
 *       + c1/h_{i+1} + c2/k_{j+1} + r
 * Fields c1, c2, r and outputs are mx*my arrays, x-fastest.
 * ---------------------------------------------------------------------- */
void orc_assemble_grid(int mx, int my, const double *xs, const double *ys, double eps,
                       const double *c1, const double *c2, const double *r,
                       double *aW, double *aE, double *aS, double *aN, double *aC)
{
    for (int j = 1; j <= my; j++) {
        double kj = ys[j] - ys[j - 1], kj1 = ys[j + 1] - ys[j];
        double kb = 0.5 * (kj + kj1);
        for (int i = 1; i <= mx; i++) {
            double hi = xs[i] - xs[i - 1], hi1 = xs[i + 1] - xs[i];
            double hb = 0.5 * (hi + hi1);
            size_t k = (size_t)(j - 1) * mx + (i - 1);
            aW[k] = -eps / (hb * hi);
            aE[k] = -eps / (hb * hi1) - c1[k] / hi1;
            aS[k] = -eps / (kb * kj);
            aN[k] = -eps / (kb * kj1) - c2[k] / kj1;
            aC[k] = eps / hb * (1.0 / hi + 1.0 / hi1) + eps / kb * (1.0 / kj + 1.0 / kj1)
                    + c1[k] / hi1 + c2[k] / kj1 + r[k];
        }
    }
}

/* Whole-domain assembly: interior nodes 1..N-1 of the Shishkin mesh. */
void orc_assemble(int N, double eps, const double *x, const double *y,
                  const double *c1, const double *c2, const double *r,
                  double *aW, double *aE, double *aS, double *aN, double *aC)
{
    orc_assemble_grid(N - 1, N - 1, x, y, eps, c1, c2, r, aW, aE, aS, aN, aC);
}

/* y = A u on an mx-by-my block with Dirichlet-0 neighbours outside it. */
static void grid_apply(int mx, int my, const double *aW, const double *aE, const double *aS,
                       const double *aN, const double *aC, const double *u, double *out)
{
    for (int j = 1; j <= my; j++)
        for (int i = 1; i <= mx; i++) {
            size_t k = (size_t)(j - 1) * mx + (i - 1);
            double s = aC[k] * u[k];
            if (i > 1) s += aW[k] * u[k - 1];
            if (i < mx) s += aE[k] * u[k + 1];
            if (j > 1) s += aS[k] * u[k - mx];
            if (j < my) s += aN[k] * u[k + mx];
            out[k] = s;
        }
}

/* y = A^T u: column (i,j) of A holds W of row (i+1,j), E of row (i-1,j),
 * S of row (i,j+1), N of row (i,j-1). */
static void grid_apply_T(int mx, int my, const double *aW, const double *aE, const double *aS,
                         const double *aN, const double *aC, const double *u, double *out)
{
    for (int j = 1; j <= my; j++)
        for (int i = 1; i <= mx; i++) {
            size_t k = (size_t)(j - 1) * mx + (i - 1);
            double s = aC[k] * u[k];
            if (i < mx) s += aW[k + 1] * u[k + 1];
            if (i > 1) s += aE[k - 1] * u[k - 1];
            if (j < my) s += aS[k + mx] * u[k + mx];
            if (j > 1) s += aN[k - mx] * u[k - mx];
            out[k] = s;
        }
}

void orc_apply(int N, const double *aW, const double *aE, const double *aS, const double *aN,
               const double *aC, const double *u, double *y, int transpose)
{
    if (transpose) grid_apply_T(N - 1, N - 1, aW, aE, aS, aN, aC, u, y);
    else grid_apply(N - 1, N - 1, aW, aE, aS, aN, aC, u, y);
}

/* ------------------------------------------------------------------------
 * O2. Banded LU without pivoting (A is an M-matrix, Sec. 3 after the stencil,
 * so Gaussian elimination without pivoting is stable).  Lower and upper
 * bandwidth N-1.  Solves A u = f, or A^T u = f when transpose != 0.
 * Memory (N-1)^2 * (2N-1) doubles.
 * ---------------------------------------------------------------------- */
int orc_band_solve(int N, const double *aW, const double *aE, const double *aS, const double *aN,
                   const double *aC, const double *f, double *u, int transpose)
{
    int M = N - 1;
    size_t n = (size_t)M * M;
    int bw = M;                 /* half bandwidth */
    int w = 2 * bw + 1;
    double *B = (double *)calloc(n * (size_t)w, sizeof(double));
    if (!B) return ORC_ERR_MEM;
#define BAND(p, q) B[(size_t)(p) * w + (size_t)((q) - (p) + bw)]
    for (int j = 1; j <= M; j++)
        for (int i = 1; i <= M; i++) {
            size_t p = ix(N, i, j);
            /* entry (row p, col q) of A; for A^T we store it at (q, p) */
#define PUT(q, v) do { if (transpose) BAND((q), (p)) = (v); else BAND((p), (q)) = (v); } while (0)
            PUT(p, aC[p]);
            if (i > 1) PUT(p - 1, aW[p]);
            if (i < M) PUT(p + 1, aE[p]);
            if (j > 1) PUT(p - M, aS[p]);
            if (j < M) PUT(p + M, aN[p]);
#undef PUT
        }
    /* Doolittle elimination, column by column. */
    for (size_t k = 0; k < n; k++) {
        double piv = BAND(k, k);
        if (piv == 0.0) { free(B); return ORC_ERR_BREAKDOWN; }
        size_t iend = k + bw < n - 1 ? k + bw : n - 1;
        size_t jend = iend;
        for (size_t i = k + 1; i <= iend; i++) {
            double l = BAND(i, k) / piv;
            if (l == 0.0) continue;
            BAND(i, k) = l;
            for (size_t jj = k + 1; jj <= jend; jj++) BAND(i, jj) -= l * BAND(k, jj);
        }
    }
    /* forward: L y = f (unit lower) */
    for (size_t i = 0; i < n; i++) {
        double s = f[i];
        size_t kbeg = i > (size_t)bw ? i - bw : 0;
        for (size_t k = kbeg; k < i; k++) s -= BAND(i, k) * u[k];
        u[i] = s;
    }
    /* backward: U u = y */
    for (size_t ii = n; ii-- > 0;) {
        double s = u[ii];
        size_t kend = ii + bw < n - 1 ? ii + bw : n - 1;
        for (size_t k = ii + 1; k <= kend; k++) s -= BAND(ii, k) * u[k];
        u[ii] = s / BAND(ii, ii);
    }
#undef BAND
    free(B);
    return ORC_OK;
}

/* Tridiagonal solve by the Thomas algorithm: sub[i] x[i-1] + dia[i] x[i] +
 * sup[i] x[i+1] = d[i], i = 0..n-1 (sub[0], sup[n-1] unused).  Used for the
 * layer-region line solves (Sec. 3.1, M_YY and M_XX: "line solves ...
 * implemented using Thomas' algorithm"). */
static void thomas(int n, const double *sub, const double *dia, const double *sup,
                   const double *d, double *x, double *cp, double *dp)
{
    cp[0] = sup[0] / dia[0];
    dp[0] = d[0] / dia[0];
    for (int i = 1; i < n; i++) {
        double den = dia[i] - sub[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? sup[i] / den : 0.0;
        dp[i] = (d[i] - sub[i] * dp[i - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* ------------------------------------------------------------------------
 * Preconditioner M of Sec. 3.1, eq. (2D blocks):
 *
 *   M = [ M_CC A_CX A_CY A_CI ;  0 M_XX A_XY A_XI ;  0 0 M_YY A_YI ;
 *         0 0 0 M_II ]
 *
 * C = [0,tau_x]x[0,tau_y] (nodes i,j <= N/2), X = [0,tau_x]x(tau_y,1]
 * (i <= N/2 < j), Y = (tau_x,1]x[0,tau_y] (j <= N/2 < i), I = the rest.
 * Applied by block back substitution: I, then Y, then X, then C.
 *
 *  M_II : upper-triangular part of A_II (keeps E and N), downstream
 *         Gauss-Seidel from the upper-right to the lower-left corner.
 *  M_YY : line solves on lines of constant x (tridiagonal in y), lines
 *         ordered right to left, keeping the E coupling to the line already
 *         solved and dropping W.
 *  M_XX : line solves on lines of constant y (tridiagonal in x), lines
 *         ordered top down, keeping the N coupling and dropping S.
 *  M_CC : Sec. 3.2, two-exponential-layer case: stationary iteration with a
 *         V(1,1) full-coarsening multigrid cycle until the corner residual
 *         has dropped by a factor `reduction` (10^3 in the paper).
 *
 * Corner multigrid (Sec. 3.2, last two paragraphs), with these readings of
 * what the paper leaves open:
 *  - level 0 is A_CC itself: nodes 1..m (m = N/2) per axis, node m is the
 *    transition point, the node m+1 outside C acts as a Dirichlet-0 node;
 *  - level l+1 keeps the even nodes of level l, so level l is the set of
 *    fine nodes with index a multiple of 2^l; the transition node is kept on
 *    every level and the outside node stays at the fine node m+1 (spacing H);
 *    coarsening stops when the side is odd or below coarsest_min*2;
 *  - coarse operators are re-discretized with the same stencil on the coarse
 *    node coordinates, with c1, c2, r injected from the coinciding fine node;
 *  - interpolation P is bilinear on the (uniform) corner mesh: weight 1/2 to a
 *    fine node between two coarse nodes on a line, 1/4 to a cell centre;
 *  - residuals are moved to finite-element scaling by D = diag(hb_i kb_j)
 *    before restriction by P^T: b_c = D_c^{-1} P^T D_f r_f;
 *  - smoother: one pointwise Gauss-Seidel sweep before and after the
 *    coarse correction, ordered from the top-right node to the bottom-left
 *    one (rows top to bottom, right to left within a row); the coarsest
 *    level gets 4 such sweeps;
 *  - the residual whose reduction stops the iteration is that of the
 *    rescaled (finite-element style) corner problem the cycle works on,
 *    D (b - A_CC e), measured in the 2-norm; at most max_cycles cycles.
 *    With this reading the stationary iteration takes the 5 cycles the paper
 *    reports for its two-exponential-layer runs.  fixed_cycles > 0 runs
 *    exactly that many cycles instead (a fixed linear operator).
 * The transpose M^T (for the adjoint solve) is block lower triangular and is
 * applied C, X, Y, I; each diagonal block is replaced by its transpose, and
 * the corner cycle by its exact transpose (forward Gauss-Seidel on A^T,
 * restriction P^T, prolongation D_f P D_c^{-1}).
 * ---------------------------------------------------------------------- */
#define ORC_MAXLEV 32
typedef struct {
    int N, m;
    double eps;
    double *x, *y;
    double *aW, *aE, *aS, *aN, *aC;   /* fine operator, n entries */
    int nlev;
    int ms[ORC_MAXLEV];
    double *lx[ORC_MAXLEV], *ly[ORC_MAXLEV];          /* coords 0..ms+1 */
    double *LW[ORC_MAXLEV], *LE[ORC_MAXLEV], *LS[ORC_MAXLEV], *LN[ORC_MAXLEV], *LC[ORC_MAXLEV];
    double *LD[ORC_MAXLEV];                             /* hb*kb */
    double *tmp_r[ORC_MAXLEV], *tmp_b[ORC_MAXLEV], *tmp_e[ORC_MAXLEV];
    double reduction;
    int max_cycles, fixed_cycles, coarsest_min;
    int corner_exact;     /* 1: M_CC = A_CC solved by banded LU (the idealised M-hat) */
    int distance;         /* 1: bilinear transfer weights from the level coordinates (graded meshes) */
    int last_cycles;
    double *wv;           /* work vectors */
    /* parabolic-layer corner cycle (semi != 0): x-semicoarsened levels of
     * width sx[l] and height m, 9-point operators A9[l] (9 planes, plane
     * (dy+1)*3 + (dx+1) holds the entry to node (I+dx, J+dy)), and the
     * interpolation weights from level l+1 to the odd columns of level l */
    int semi, snlev;
    int sx[ORC_MAXLEV];
    double *A9[ORC_MAXLEV], *PW[ORC_MAXLEV], *PE[ORC_MAXLEV];
    double *sr[ORC_MAXLEV], *sb[ORC_MAXLEV], *se[ORC_MAXLEV];
} orc_prec;

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

void orc_prec_destroy(orc_prec *P)
{
    if (!P) return;
    free(P->x); free(P->y);
    free(P->aW); free(P->aE); free(P->aS); free(P->aN); free(P->aC);
    for (int l = 0; l < P->nlev; l++) {
        free(P->lx[l]); free(P->ly[l]);
        free(P->LW[l]); free(P->LE[l]); free(P->LS[l]); free(P->LN[l]); free(P->LC[l]);
        free(P->LD[l]); free(P->tmp_r[l]); free(P->tmp_b[l]); free(P->tmp_e[l]);
    }
    for (int l = 0; l < P->snlev; l++) {
        free(P->A9[l]); free(P->PW[l]); free(P->PE[l]); free(P->sr[l]); free(P->sb[l]); free(P->se[l]);
    }
    free(P->wv);
    free(P);
}

static void semi_build(orc_prec *P);

/* The block split of Sec. 3.1 at layer index NL: layer set {1..NL} per axis
 * (NL = N/2 on the mesh of Sec. 3; any NL for the general mesh of the
 * Remark on general Shishkin meshes, whose analysis allows any number of
 * layer and interior points). */
orc_prec *orc_prec_create_split(int N, int NL, double eps, const double *x, const double *y,
                                const double *c1, const double *c2, const double *r,
                                double reduction, int max_cycles, int fixed_cycles, int coarsest_min,
                                int corner_exact, int semi)
{
    if (N < 4 || NL < 1 || NL > N - 2 || (semi && NL != N / 2)) return NULL;
    orc_prec *P = (orc_prec *)calloc(1, sizeof(orc_prec));
    int M = N - 1, m = NL;
    size_t n = (size_t)M * M;
    P->N = N; P->m = m; P->eps = eps;
    P->reduction = reduction; P->max_cycles = max_cycles; P->fixed_cycles = fixed_cycles;
    P->coarsest_min = coarsest_min < 1 ? 1 : coarsest_min;
    P->corner_exact = corner_exact;
    P->x = dalloc(N + 1); P->y = dalloc(N + 1);
    memcpy(P->x, x, sizeof(double) * (N + 1));
    memcpy(P->y, y, sizeof(double) * (N + 1));
    P->aW = dalloc(n); P->aE = dalloc(n); P->aS = dalloc(n); P->aN = dalloc(n); P->aC = dalloc(n);
    orc_assemble(N, eps, x, y, c1, c2, r, P->aW, P->aE, P->aS, P->aN, P->aC);
    P->wv = dalloc(8 * (size_t)N + 16);

    /* corner levels */
    int ml = m, l = 0;
    for (;;) {
        int stride = 1 << l;
        P->ms[l] = ml;
        size_t nl = (size_t)ml * ml;
        P->lx[l] = dalloc(ml + 2); P->ly[l] = dalloc(ml + 2);
        P->lx[l][0] = x[0]; P->ly[l][0] = y[0];
        for (int I = 1; I <= ml; I++) { P->lx[l][I] = x[I * stride]; P->ly[l][I] = y[I * stride]; }
        P->lx[l][ml + 1] = x[m + 1]; P->ly[l][ml + 1] = y[m + 1];
        double *f1 = dalloc(nl), *f2 = dalloc(nl), *fr = dalloc(nl);
        for (int J = 1; J <= ml; J++)
            for (int I = 1; I <= ml; I++) {
                size_t kf = ix(N, I * stride, J * stride), kc = (size_t)(J - 1) * ml + (I - 1);
                f1[kc] = c1[kf]; f2[kc] = c2[kf]; fr[kc] = r[kf];
            }
        P->LW[l] = dalloc(nl); P->LE[l] = dalloc(nl); P->LS[l] = dalloc(nl);
        P->LN[l] = dalloc(nl); P->LC[l] = dalloc(nl); P->LD[l] = dalloc(nl);
        orc_assemble_grid(ml, ml, P->lx[l], P->ly[l], eps, f1, f2, fr,
                          P->LW[l], P->LE[l], P->LS[l], P->LN[l], P->LC[l]);
        for (int J = 1; J <= ml; J++)
            for (int I = 1; I <= ml; I++) {
                double hb = 0.5 * (P->lx[l][I + 1] - P->lx[l][I - 1]);
                double kb = 0.5 * (P->ly[l][J + 1] - P->ly[l][J - 1]);
                P->LD[l][(size_t)(J - 1) * ml + (I - 1)] = hb * kb;
            }
        free(f1); free(f2); free(fr);
        P->tmp_r[l] = dalloc(nl); P->tmp_b[l] = dalloc(nl); P->tmp_e[l] = dalloc(nl);
        l++;
        if ((ml & 1) || ml / 2 < P->coarsest_min || ml < 4 || l >= ORC_MAXLEV) break;
        ml /= 2;
    }
    P->nlev = l;
    P->semi = semi;
    if (semi) semi_build(P);
    return P;
}

orc_prec *orc_prec_create(int N, double eps, const double *x, const double *y,
                          const double *c1, const double *c2, const double *r,
                          double reduction, int max_cycles, int fixed_cycles, int coarsest_min,
                          int corner_exact, int semi)
{
    if (N < 4 || (N & 1)) return NULL;
    return orc_prec_create_split(N, N / 2, eps, x, y, c1, c2, r, reduction, max_cycles, fixed_cycles,
                                 coarsest_min, corner_exact, semi);
}

/* Choose the transfer weights of the full-coarsening corner cycle: 0 the
 * index weights of Sec. 3.2 (1/2, 1/4), 1 linear interpolation in the level
 * coordinates (the same on the uniform corner of the mesh of Sec. 3). */
void orc_prec_set_distance(orc_prec *P, int distance) { P->distance = distance; }

int orc_prec_nlev(const orc_prec *P) { return P->nlev; }
int orc_prec_level_size(const orc_prec *P, int l) { return P->ms[l]; }
int orc_prec_last_cycles(const orc_prec *P) { return P->last_cycles; }

/* Copy out the level-l corner operator and its coordinates (for tests). */
void orc_prec_level(const orc_prec *P, int l, double *xs, double *ys, double *W, double *E,
                    double *S, double *Nn, double *C, double *D)
{
    int ml = P->ms[l];
    size_t nl = (size_t)ml * ml;
    memcpy(xs, P->lx[l], sizeof(double) * (ml + 2));
    memcpy(ys, P->ly[l], sizeof(double) * (ml + 2));
    memcpy(W, P->LW[l], nl * sizeof(double)); memcpy(E, P->LE[l], nl * sizeof(double));
    memcpy(S, P->LS[l], nl * sizeof(double)); memcpy(Nn, P->LN[l], nl * sizeof(double));
    memcpy(C, P->LC[l], nl * sizeof(double)); memcpy(D, P->LD[l], nl * sizeof(double));
}

/* Downstream pointwise Gauss-Seidel sweep on level l: rows from top to
 * bottom, right to left in each row (Sec. 3.2).  transpose: the sweep of the
 * transposed cycle, i.e. forward Gauss-Seidel on A^T, bottom-left first. */
void orc_mg_gs(orc_prec *P, int l, const double *b, double *e, int transpose)
{
    int ml = P->ms[l];
    const double *W = P->LW[l], *E = P->LE[l], *S = P->LS[l], *Nn = P->LN[l], *C = P->LC[l];
    if (!transpose) {
        for (int J = ml; J >= 1; J--)
            for (int I = ml; I >= 1; I--) {
                size_t k = (size_t)(J - 1) * ml + (I - 1);
                double s = b[k];
                if (I > 1) s -= W[k] * e[k - 1];
                if (I < ml) s -= E[k] * e[k + 1];
                if (J > 1) s -= S[k] * e[k - ml];
                if (J < ml) s -= Nn[k] * e[k + ml];
                e[k] = s / C[k];
            }
    } else {
        for (int J = 1; J <= ml; J++)
            for (int I = 1; I <= ml; I++) {
                size_t k = (size_t)(J - 1) * ml + (I - 1);
                double s = b[k];
                if (I < ml) s -= W[k + 1] * e[k + 1];
                if (I > 1) s -= E[k - 1] * e[k - 1];
                if (J < ml) s -= S[k + ml] * e[k + ml];
                if (J > 1) s -= Nn[k - ml] * e[k - ml];
                e[k] = s / C[k];
            }
    }
}

/* Bilinear interpolation from level l+1 (side mc) to level l (side mf):
 * ef += P ec.  Fine node (I,J) with I,J even coincides with coarse node
 * (I/2,J/2); odd indices take the two (or four) surrounding coarse nodes;
 * coarse index 0 is the Dirichlet boundary (value 0).  The 1D weights of an
 * odd fine index I are 1/2, 1/2 on the mesh of Sec. 3 (uniform in the
 * corner), or, with P->distance, the distances to the two coarse nodes:
 * (x_{I+1} - x_I) / (x_{I+1} - x_{I-1}) for coarse node (I-1)/2 and
 * (x_I - x_{I-1}) / (x_{I+1} - x_{I-1}) for (I+1)/2 (the level-l coordinates),
 * which is linear interpolation on a non-uniform (graded) mesh. */
static double coarse_at(const double *ec, int mc, int I, int J)
{
    if (I < 1 || J < 1 || I > mc || J > mc) return 0.0;
    return ec[(size_t)(J - 1) * mc + (I - 1)];
}
/* weights of the coarse nodes to the left and right of odd fine index I */
static void lin_weights(const orc_prec *P, const double *c, int I, double *wl, double *wr)
{
    if (!P->distance) { *wl = 0.5; *wr = 0.5; return; }
    double d = c[I + 1] - c[I - 1];
    *wl = (c[I + 1] - c[I]) / d;
    *wr = (c[I] - c[I - 1]) / d;
}
void orc_mg_prolong(orc_prec *P, int l, const double *ec, double *ef)
{
    int mf = P->ms[l], mc = P->ms[l + 1];
    const double *cx = P->lx[l], *cy = P->ly[l];
    for (int J = 1; J <= mf; J++)
        for (int I = 1; I <= mf; I++) {
            double v, ax = 1.0, bx = 0.0, ay = 1.0, by = 0.0;
            int Ie = !(I & 1), Je = !(J & 1);
            if (!Ie) lin_weights(P, cx, I, &ax, &bx);
            if (!Je) lin_weights(P, cy, J, &ay, &by);
            if (Ie && Je) v = coarse_at(ec, mc, I / 2, J / 2);
            else if (!Ie && Je) v = ax * coarse_at(ec, mc, (I - 1) / 2, J / 2) + bx * coarse_at(ec, mc, (I + 1) / 2, J / 2);
            else if (Ie && !Je) v = ay * coarse_at(ec, mc, I / 2, (J - 1) / 2) + by * coarse_at(ec, mc, I / 2, (J + 1) / 2);
            else if (!P->distance)
                v = 0.25 * (coarse_at(ec, mc, (I - 1) / 2, (J - 1) / 2) + coarse_at(ec, mc, (I + 1) / 2, (J - 1) / 2)
                            + coarse_at(ec, mc, (I - 1) / 2, (J + 1) / 2) + coarse_at(ec, mc, (I + 1) / 2, (J + 1) / 2));
            else
                v = ay * (ax * coarse_at(ec, mc, (I - 1) / 2, (J - 1) / 2) + bx * coarse_at(ec, mc, (I + 1) / 2, (J - 1) / 2))
                    + by * (ax * coarse_at(ec, mc, (I - 1) / 2, (J + 1) / 2) + bx * coarse_at(ec, mc, (I + 1) / 2, (J + 1) / 2));
            ef[(size_t)(J - 1) * mf + (I - 1)] += v;
        }
}

/* bc = P^T rf (transpose of orc_mg_prolong), written as a plain scatter. */
static void prolong_T(const orc_prec *P, int l, const double *rf, double *bc)
{
    int mf = P->ms[l], mc = P->ms[l + 1];
    const double *cx = P->lx[l], *cy = P->ly[l];
    for (size_t k = 0; k < (size_t)mc * mc; k++) bc[k] = 0.0;
    for (int J = 1; J <= mf; J++)
        for (int I = 1; I <= mf; I++) {
            double v = rf[(size_t)(J - 1) * mf + (I - 1)];
            double ax = 1.0, bx = 0.0, ay = 1.0, by = 0.0;
            int Ie = !(I & 1), Je = !(J & 1);
            if (!Ie) lin_weights(P, cx, I, &ax, &bx);
            if (!Je) lin_weights(P, cy, J, &ay, &by);
#define ADD(Ic, Jc, w) do { int _I = (Ic), _J = (Jc); if (_I >= 1 && _J >= 1 && _I <= mc && _J <= mc) bc[(size_t)(_J - 1) * mc + (_I - 1)] += (w) * v; } while (0)
            if (Ie && Je) ADD(I / 2, J / 2, 1.0);
            else if (!Ie && Je) { ADD((I - 1) / 2, J / 2, ax); ADD((I + 1) / 2, J / 2, bx); }
            else if (Ie && !Je) { ADD(I / 2, (J - 1) / 2, ay); ADD(I / 2, (J + 1) / 2, by); }
            else if (!P->distance) {
                ADD((I - 1) / 2, (J - 1) / 2, 0.25); ADD((I + 1) / 2, (J - 1) / 2, 0.25);
                ADD((I - 1) / 2, (J + 1) / 2, 0.25); ADD((I + 1) / 2, (J + 1) / 2, 0.25);
            } else {
                ADD((I - 1) / 2, (J - 1) / 2, ax * ay); ADD((I + 1) / 2, (J - 1) / 2, bx * ay);
                ADD((I - 1) / 2, (J + 1) / 2, ax * by); ADD((I + 1) / 2, (J + 1) / 2, bx * by);
            }
#undef ADD
        }
}

/* Restriction of a level-l residual to level l+1: bc = D_c^{-1} P^T D_f rf
 * (forward cycle), or bc = P^T rf (transposed cycle). */
void orc_mg_restrict(orc_prec *P, int l, const double *rf, double *bc, int transpose)
{
    int mf = P->ms[l], mc = P->ms[l + 1];
    size_t nf = (size_t)mf * mf, nc = (size_t)mc * mc;
    if (!transpose) {
        double *t = dalloc(nf);
        for (size_t k = 0; k < nf; k++) t[k] = P->LD[l][k] * rf[k];
        prolong_T(P, l, t, bc);
        for (size_t k = 0; k < nc; k++) bc[k] /= P->LD[l + 1][k];
        free(t);
    } else {
        prolong_T(P, l, rf, bc);
    }
}

/* One V(1,1) cycle on level l for A_l e = b, improving e in place. */
void orc_mg_vcycle(orc_prec *P, int l, const double *b, double *e, int transpose)
{
    int ml = P->ms[l];
    size_t nl = (size_t)ml * ml;
    if (l == P->nlev - 1) {
        for (int s = 0; s < 4; s++) orc_mg_gs(P, l, b, e, transpose);
        return;
    }
    orc_mg_gs(P, l, b, e, transpose);
    double *r = P->tmp_r[l];
    if (transpose) grid_apply_T(ml, ml, P->LW[l], P->LE[l], P->LS[l], P->LN[l], P->LC[l], e, r);
    else grid_apply(ml, ml, P->LW[l], P->LE[l], P->LS[l], P->LN[l], P->LC[l], e, r);
    for (size_t k = 0; k < nl; k++) r[k] = b[k] - r[k];
    int mc = P->ms[l + 1];
    size_t nc = (size_t)mc * mc;
    double *bc = P->tmp_b[l + 1], *ec = P->tmp_e[l + 1];
    orc_mg_restrict(P, l, r, bc, transpose);
    for (size_t k = 0; k < nc; k++) ec[k] = 0.0;
    orc_mg_vcycle(P, l + 1, bc, ec, transpose);
    if (!transpose) {
        orc_mg_prolong(P, l, ec, e);
    } else {
        /* prolongation of the transposed cycle: R^T = D_f P D_c^{-1} */
        double *t = dalloc(nc), *pf = dalloc(nl);
        for (size_t k = 0; k < nc; k++) t[k] = ec[k] / P->LD[l + 1][k];
        orc_mg_prolong(P, l, t, pf);
        for (size_t k = 0; k < nl; k++) e[k] += P->LD[l][k] * pf[k];
        free(t); free(pf);
    }
    orc_mg_gs(P, l, b, e, transpose);
}

static double nrm2(size_t n, const double *v)
{
    double s = 0.0;
    for (size_t k = 0; k < n; k++) s += v[k] * v[k];
    return sqrt(s);
}

/* ------------------------------------------------------------------------
 * Corner multigrid for one parabolic and one exponential layer (Sec. 3.2,
 * the case of eq. (tau parabolic)), taken step by step as the paper states
 * it:
 *  - inside the cycle the corner rows are rescaled to finite-element size,
 *    row (x_i, y_j) of A_CC multiplied by hb_i kb_j, and the residual with
 *    it: the cycle works on A_0 = D A_CC, D b;
 *  - coarse levels coarsen by 2 in x only: coarse column I is fine column
 *    2I, every row is kept; coarsening continues while the width is even,
 *    at least 4, and half of it is at least coarsest_min;
 *  - interpolation is induced by the operator: row (i,j) of the level
 *    matrix is collapsed North-South, and an odd fine column i takes from
 *    coarse columns (i-1)/2 and (i+1)/2 (same row) the weights
 *        -(a[(i,j),(i-1,j-1)] + a[(i,j),(i-1,j)] + a[(i,j),(i-1,j+1)]) / s,
 *        -(a[(i,j),(i+1,j-1)] + a[(i,j),(i+1,j)] + a[(i,j),(i+1,j+1)]) / s,
 *        s = a[(i,j),(i,j-1)] + a[(i,j),(i,j)] + a[(i,j),(i,j+1)];
 *    even columns are injected.  Only entries of the matrix enter the sums:
 *    couplings to nodes outside the block (the boundary, the X and Y
 *    regions) are not entries of A_CC and count as 0;
 *  - restriction is P^T and each coarse operator the Galerkin product
 *    A_{l+1} = P^T A_l P (nine-point on every coarse level);
 *  - relaxation is pointwise Gauss-Seidel in the downstream order (rows top
 *    to bottom, right to left within a row), V(1,1), four sweeps on the
 *    coarsest level;
 *  - cycles run until ||D b - A_0 e||_2 <= ||D b||_2 / reduction (the paper
 *    uses 10^2 for this case), at most max_cycles, or fixed_cycles exactly.
 * Only the forward cycle is provided.
 * ---------------------------------------------------------------------- */
static size_t plane(int dx, int dy) { return (size_t)((dy + 1) * 3 + (dx + 1)); }

/* entry of the level-l matrix in row (I,J), column (I+dx, J+dy); 0 when that
 * node is outside the level's block */
static double semi_a(const orc_prec *P, int l, int I, int J, int dx, int dy)
{
    int sx = P->sx[l], m = P->m;
    if (I + dx < 1 || I + dx > sx || J + dy < 1 || J + dy > m) return 0.0;
    return P->A9[l][plane(dx, dy) * ((size_t)sx * m) + (size_t)(J - 1) * sx + (I - 1)];
}

/* the coarse columns (level l+1, same row) that fine node (I,J) of level l
 * interpolates from, with their weights; returns how many */
static int semi_pcols(const orc_prec *P, int l, int I, int J, int *Ic, double *w)
{
    if (!(I & 1)) { Ic[0] = I / 2; w[0] = 1.0; return 1; }
    size_t k = (size_t)(J - 1) * P->sx[l] + (I - 1);
    int c = 0;
    if ((I - 1) / 2 >= 1) { Ic[c] = (I - 1) / 2; w[c] = P->PW[l][k]; c++; }
    if ((I + 1) / 2 <= P->sx[l + 1]) { Ic[c] = (I + 1) / 2; w[c] = P->PE[l][k]; c++; }
    return c;
}

static void semi_weights(orc_prec *P, int l)
{
    int sx = P->sx[l], m = P->m;
    size_t n = (size_t)sx * m;
    P->PW[l] = dalloc(n); P->PE[l] = dalloc(n);
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= sx; I += 2) {
            double s = semi_a(P, l, I, J, 0, -1) + semi_a(P, l, I, J, 0, 0) + semi_a(P, l, I, J, 0, 1);
            double w = semi_a(P, l, I, J, -1, -1) + semi_a(P, l, I, J, -1, 0) + semi_a(P, l, I, J, -1, 1);
            double e = semi_a(P, l, I, J, 1, -1) + semi_a(P, l, I, J, 1, 0) + semi_a(P, l, I, J, 1, 1);
            size_t k = (size_t)(J - 1) * sx + (I - 1);
            P->PW[l][k] = -w / s;
            P->PE[l][k] = -e / s;
        }
}

/* A_{l+1} = P^T A_l P: sum over fine rows p and their nonzero entries
 * a = A_l[p,q] of P[p,c1] a P[q,c2] into A_{l+1}[c1,c2] */
static void semi_galerkin(orc_prec *P, int l)
{
    int sx = P->sx[l], sxc = P->sx[l + 1], m = P->m;
    size_t nc = (size_t)sxc * m;
    double *Ac = P->A9[l + 1];
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= sx; I++) {
            int Ip[2], Iq[2];
            double wp[2], wq[2];
            int np_ = semi_pcols(P, l, I, J, Ip, wp);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    double a = semi_a(P, l, I, J, dx, dy);
                    if (a == 0.0) continue;
                    int nq = semi_pcols(P, l, I + dx, J + dy, Iq, wq);
                    for (int s = 0; s < np_; s++)
                        for (int t = 0; t < nq; t++) {
                            int ddx = Iq[t] - Ip[s];
                            if (ddx < -1 || ddx > 1) continue;   /* cannot happen: P spans one coarse column each side */
                            Ac[plane(ddx, dy) * nc + (size_t)(J - 1) * sxc + (Ip[s] - 1)] += wp[s] * a * wq[t];
                        }
                }
        }
}

static void semi_build(orc_prec *P)
{
    int m = P->m, sx = m;
    size_t n = (size_t)m * m;
    P->sx[0] = m;
    P->A9[0] = dalloc(9 * n);
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= m; I++) {
            size_t k = (size_t)(J - 1) * m + (I - 1);
            double d = P->LD[0][k];
            P->A9[0][plane(0, 0) * n + k] = d * P->LC[0][k];
            if (I > 1) P->A9[0][plane(-1, 0) * n + k] = d * P->LW[0][k];
            if (I < m) P->A9[0][plane(1, 0) * n + k] = d * P->LE[0][k];
            if (J > 1) P->A9[0][plane(0, -1) * n + k] = d * P->LS[0][k];
            if (J < m) P->A9[0][plane(0, 1) * n + k] = d * P->LN[0][k];
        }
    int l = 0;
    for (;;) {
        size_t nl = (size_t)P->sx[l] * m;
        P->sr[l] = dalloc(nl); P->sb[l] = dalloc(nl); P->se[l] = dalloc(nl);
        if ((sx & 1) || sx / 2 < P->coarsest_min || sx < 4 || l + 1 >= ORC_MAXLEV) break;
        semi_weights(P, l);
        sx /= 2;
        P->sx[l + 1] = sx;
        P->A9[l + 1] = dalloc(9 * (size_t)sx * m);
        semi_galerkin(P, l);
        l++;
    }
    P->snlev = l + 1;
}

static void semi_apply(const orc_prec *P, int l, const double *e, double *out)
{
    int sx = P->sx[l], m = P->m;
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= sx; I++) {
            double s = 0.0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    double a = semi_a(P, l, I, J, dx, dy);
                    if (a != 0.0) s += a * e[(size_t)(J + dy - 1) * sx + (I + dx - 1)];
                }
            out[(size_t)(J - 1) * sx + (I - 1)] = s;
        }
}

void orc_semi_gs(orc_prec *P, int l, const double *b, double *e)
{
    int sx = P->sx[l], m = P->m;
    for (int J = m; J >= 1; J--)
        for (int I = sx; I >= 1; I--) {
            double s = b[(size_t)(J - 1) * sx + (I - 1)];
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (!dx && !dy) continue;
                    double a = semi_a(P, l, I, J, dx, dy);
                    if (a != 0.0) s -= a * e[(size_t)(J + dy - 1) * sx + (I + dx - 1)];
                }
            e[(size_t)(J - 1) * sx + (I - 1)] = s / semi_a(P, l, I, J, 0, 0);
        }
}

/* ef += P ec (level l+1 to level l) and bc = P^T rf */
static void semi_prolong(const orc_prec *P, int l, const double *ec, double *ef)
{
    int sx = P->sx[l], sxc = P->sx[l + 1], m = P->m;
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= sx; I++) {
            int Ic[2];
            double w[2];
            int c = semi_pcols(P, l, I, J, Ic, w);
            for (int t = 0; t < c; t++) ef[(size_t)(J - 1) * sx + (I - 1)] += w[t] * ec[(size_t)(J - 1) * sxc + (Ic[t] - 1)];
        }
}
static void semi_restrict(const orc_prec *P, int l, const double *rf, double *bc)
{
    int sx = P->sx[l], sxc = P->sx[l + 1], m = P->m;
    for (size_t k = 0; k < (size_t)sxc * m; k++) bc[k] = 0.0;
    for (int J = 1; J <= m; J++)
        for (int I = 1; I <= sx; I++) {
            int Ic[2];
            double w[2];
            int c = semi_pcols(P, l, I, J, Ic, w);
            for (int t = 0; t < c; t++) bc[(size_t)(J - 1) * sxc + (Ic[t] - 1)] += w[t] * rf[(size_t)(J - 1) * sx + (I - 1)];
        }
}

static void semi_vcycle(orc_prec *P, int l, const double *b, double *e)
{
    if (l == P->snlev - 1) {
        for (int s = 0; s < 4; s++) orc_semi_gs(P, l, b, e);
        return;
    }
    size_t nl = (size_t)P->sx[l] * P->m, nc = (size_t)P->sx[l + 1] * P->m;
    double *r = P->sr[l], *bc = P->sb[l + 1], *ec = P->se[l + 1];
    orc_semi_gs(P, l, b, e);
    semi_apply(P, l, e, r);
    for (size_t k = 0; k < nl; k++) r[k] = b[k] - r[k];
    semi_restrict(P, l, r, bc);
    for (size_t k = 0; k < nc; k++) ec[k] = 0.0;
    semi_vcycle(P, l + 1, bc, ec);
    semi_prolong(P, l, ec, e);
    orc_semi_gs(P, l, b, e);
}

static int semi_corner_solve(orc_prec *P, const double *b, double *e)
{
    int m = P->m;
    size_t nc = (size_t)m * m;
    double *bs = dalloc(nc), *r = dalloc(nc);
    for (size_t k = 0; k < nc; k++) { bs[k] = P->LD[0][k] * b[k]; e[k] = 0.0; }
    double b0 = nrm2(nc, bs);
    int cyc = 0;
    while (b0 > 0.0) {
        if (P->fixed_cycles > 0 ? cyc >= P->fixed_cycles : cyc >= P->max_cycles) break;
        semi_vcycle(P, 0, bs, e);
        cyc++;
        if (P->fixed_cycles <= 0) {
            semi_apply(P, 0, e, r);
            for (size_t k = 0; k < nc; k++) r[k] = bs[k] - r[k];
            if (nrm2(nc, r) <= b0 / P->reduction) break;
        }
    }
    free(bs); free(r);
    return cyc;
}

/* level data of the parabolic cycle, for the tests: the nine planes of A_l
 * (9 * width * m values, plane (dy+1)*3 + (dx+1)) and, below the coarsest
 * level, the interpolation weights of the odd columns (0 elsewhere) */
int orc_semi_nlev(const orc_prec *P) { return P->semi ? P->snlev : 0; }
int orc_semi_width(const orc_prec *P, int l) { return P->sx[l]; }
void orc_semi_level(const orc_prec *P, int l, double *A9, double *PW, double *PE)
{
    size_t n = (size_t)P->sx[l] * P->m;
    memcpy(A9, P->A9[l], 9 * n * sizeof(double));
    if (l < P->snlev - 1) { memcpy(PW, P->PW[l], n * sizeof(double)); memcpy(PE, P->PE[l], n * sizeof(double)); }
}

/* M_CC^{-1} b (or M_CC^{-T} b): stationary multigrid iteration from e = 0.
 * Returns the number of cycles taken. */
int orc_corner_solve(orc_prec *P, const double *b, double *e, int transpose)
{
    int m = P->m;
    size_t nc = (size_t)m * m;
    for (size_t k = 0; k < nc; k++) e[k] = 0.0;
    if (P->semi) return transpose ? -1 : semi_corner_solve(P, b, e);
    if (P->corner_exact) {
        /* the idealised M-hat of Sec. 3.1: exact A_CC solve (banded LU on the
         * corner block, which is the level-0 operator) */
        int rc = orc_band_solve(m + 1, P->LW[0], P->LE[0], P->LS[0], P->LN[0], P->LC[0], b, e, transpose);
        (void)rc;
        return 0;
    }
    double *r = dalloc(nc);
    const double *D = P->LD[0];
    for (size_t k = 0; k < nc; k++) r[k] = D[k] * b[k];
    double b0 = nrm2(nc, r);
    int cyc = 0;
    if (b0 == 0.0) { free(r); return 0; }
    for (;;) {
        if (P->fixed_cycles > 0 && cyc >= P->fixed_cycles) break;
        if (P->fixed_cycles <= 0 && cyc >= P->max_cycles) break;
        orc_mg_vcycle(P, 0, b, e, transpose);
        cyc++;
        if (P->fixed_cycles <= 0) {
            if (transpose) grid_apply_T(m, m, P->LW[0], P->LE[0], P->LS[0], P->LN[0], P->LC[0], e, r);
            else grid_apply(m, m, P->LW[0], P->LE[0], P->LS[0], P->LN[0], P->LC[0], e, r);
            for (size_t k = 0; k < nc; k++) r[k] = D[k] * (b[k] - r[k]);
            if (nrm2(nc, r) <= b0 / P->reduction) break;
        }
    }
    free(r);
    return cyc;
}

/* z = M^{-1} v (transpose = 0) or z = M^{-T} v (transpose = 1), whole domain.
 * Returns the number of corner cycles used. */
int orc_prec_apply(orc_prec *P, const double *v, double *z, int transpose)
{
    int N = P->N, m = P->m, M = N - 1;
    const double *aW = P->aW, *aE = P->aE, *aS = P->aS, *aN = P->aN, *aC = P->aC;
    double *sub = P->wv, *dia = sub + N, *sup = dia + N, *rhs = sup + N, *sol = rhs + N,
           *cp = sol + N, *dp = cp + N;
    size_t n = (size_t)M * M;
    for (size_t k = 0; k < n; k++) z[k] = 0.0;
    int L = m;          /* last layer index (transition node) */
    int cyc = 0;
    size_t nc = (size_t)m * m;
    double *bc = dalloc(nc), *ec = dalloc(nc);

    if (!transpose) {
        /* I block: M_II z_I = v_I, sweep from (N-1,N-1) down to (L+1,L+1) */
        for (int j = M; j >= L + 1; j--)
            for (int i = M; i >= L + 1; i--) {
                size_t k = ix(N, i, j);
                double s = v[k];
                if (i < M) s -= aE[k] * z[k + 1];
                if (j < M) s -= aN[k] * z[k + M];
                z[k] = s / aC[k];
            }
        /* Y block: lines of constant x, i = N-1 down to L+1, j = 1..L */
        for (int i = M; i >= L + 1; i--) {
            for (int j = 1; j <= L; j++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                if (i < M) s -= aE[k] * z[k + 1];        /* E coupling (line i+1, in Y) */
                if (j == L) s -= aN[k] * z[k + M];       /* A_YI: north neighbour in I */
                rhs[j - 1] = s;
                sub[j - 1] = aS[k]; dia[j - 1] = aC[k]; sup[j - 1] = aN[k];
            }
            thomas(L, sub, dia, sup, rhs, sol, cp, dp);
            for (int j = 1; j <= L; j++) z[ix(N, i, j)] = sol[j - 1];
        }
        /* X block: lines of constant y, j = N-1 down to L+1, i = 1..L */
        for (int j = M; j >= L + 1; j--) {
            for (int i = 1; i <= L; i++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                if (j < M) s -= aN[k] * z[k + M];        /* N coupling (line j+1, in X) */
                if (i == L) s -= aE[k] * z[k + 1];       /* A_XI: east neighbour in I */
                rhs[i - 1] = s;
                sub[i - 1] = aW[k]; dia[i - 1] = aC[k]; sup[i - 1] = aE[k];
            }
            thomas(L, sub, dia, sup, rhs, sol, cp, dp);
            for (int i = 1; i <= L; i++) z[ix(N, i, j)] = sol[i - 1];
        }
        /* C block: b_C = v_C - A_CX z_X - A_CY z_Y, then M_CC^{-1} */
        for (int j = 1; j <= L; j++)
            for (int i = 1; i <= L; i++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                if (j == L) s -= aN[k] * z[k + M];       /* A_CX */
                if (i == L) s -= aE[k] * z[k + 1];       /* A_CY */
                bc[(size_t)(j - 1) * m + (i - 1)] = s;
            }
        cyc = orc_corner_solve(P, bc, ec, 0);
        for (int j = 1; j <= L; j++)
            for (int i = 1; i <= L; i++) z[ix(N, i, j)] = ec[(size_t)(j - 1) * m + (i - 1)];
    } else {
        /* M^T is block lower triangular: C, then X, then Y, then I. */
        for (int j = 1; j <= L; j++)
            for (int i = 1; i <= L; i++) bc[(size_t)(j - 1) * m + (i - 1)] = v[ix(N, i, j)];
        cyc = orc_corner_solve(P, bc, ec, 1);
        for (int j = 1; j <= L; j++)
            for (int i = 1; i <= L; i++) z[ix(N, i, j)] = ec[(size_t)(j - 1) * m + (i - 1)];
        /* X^T: lines j = L+1 .. N-1 (bottom up), T_j^T along x */
        for (int j = L + 1; j <= M; j++) {
            for (int i = 1; i <= L; i++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                /* coupling from the line below: row (i,j) of M^T holds N of (i,j-1);
                 * for j = L+1 that node is in C (A_CX^T), otherwise in X */
                s -= aN[k - M] * z[k - M];
                rhs[i - 1] = s;
                sub[i - 1] = (i > 1) ? aE[k - 1] : 0.0;   /* (T^T)_{i,i-1} = T_{i-1,i} = E of i-1 */
                dia[i - 1] = aC[k];
                sup[i - 1] = (i < L) ? aW[k + 1] : 0.0;   /* (T^T)_{i,i+1} = W of i+1 */
            }
            thomas(L, sub, dia, sup, rhs, sol, cp, dp);
            for (int i = 1; i <= L; i++) z[ix(N, i, j)] = sol[i - 1];
        }
        /* Y^T: lines i = L+1 .. N-1 (left to right), T_i^T along y */
        for (int i = L + 1; i <= M; i++) {
            for (int j = 1; j <= L; j++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                s -= aE[k - 1] * z[k - 1];            /* from line i-1 (Y) or C (A_CY^T) */
                rhs[j - 1] = s;
                sub[j - 1] = (j > 1) ? aN[k - M] : 0.0;
                dia[j - 1] = aC[k];
                sup[j - 1] = (j < L) ? aS[k + M] : 0.0;
            }
            thomas(L, sub, dia, sup, rhs, sol, cp, dp);
            for (int j = 1; j <= L; j++) z[ix(N, i, j)] = sol[j - 1];
        }
        /* I^T: forward sweep from (L+1,L+1) to (N-1,N-1); the W neighbour at
         * i = L+1 is in X (A_XI^T), the S neighbour at j = L+1 is in Y (A_YI^T) */
        for (int j = L + 1; j <= M; j++)
            for (int i = L + 1; i <= M; i++) {
                size_t k = ix(N, i, j);
                double s = v[k];
                s -= aE[k - 1] * z[k - 1];
                s -= aN[k - M] * z[k - M];
                z[k] = s / aC[k];
            }
    }
    free(bc); free(ec);
    P->last_cycles = cyc;
    return cyc;
}

/* ------------------------------------------------------------------------
 * O3. Restarted flexible GMRES (Saad), right preconditioned, modified
 * Gram-Schmidt Arnoldi (Sec. 3.3: FGMRES, MGS/Arnoldi, solution built once
 * converged).  P == NULL gives unpreconditioned GMRES.  Stops when the true
 * residual ||S(f - A u)||_2 <= tol * (tol_abs ? 1 : ||S f||_2), S = I or,
 * with scaled != 0, S = diag(A)^{-1} (the row-normalised system, whose FP64
 * rounding floor stays near 1e-14 where the unscaled residual's does not).
 * u holds the initial guess on entry.  transpose solves A^T u = f with M^T.
 * ---------------------------------------------------------------------- */
/* Operator of the (optionally row-scaled) system: out = S A u with S = I,
 * or S = diag(A)^{-1} when scaled (row scaling of A, and of A^T's rows
 * when transpose, i.e. diag(A)^{-1} A^T). */
static void sys_apply(int N, const double *aW, const double *aE, const double *aS, const double *aN,
                      const double *aC, const double *u, double *out, int transpose, int scaled)
{
    size_t n = (size_t)(N - 1) * (N - 1);
    orc_apply(N, aW, aE, aS, aN, aC, u, out, transpose);
    if (scaled) for (size_t k = 0; k < n; k++) out[k] /= aC[k];
}

int orc_fgmres(orc_prec *P, int N, const double *aW, const double *aE, const double *aS,
               const double *aN, const double *aC, const double *f, double *u, double tol,
               int tol_abs, int restart, int maxit, int transpose, int scaled, int *iters_out,
               double *relres_out, int *max_cycles_out)
{
    int M = N - 1;
    size_t n = (size_t)M * M;
    int mr = restart;
    double *V = dalloc(n * (mr + 1)), *Z = dalloc(n * mr), *w = dalloc(n), *fs = dalloc(n), *t = dalloc(n);
    double *H = dalloc((size_t)(mr + 1) * mr), *cs = dalloc(mr), *sn = dalloc(mr), *g = dalloc(mr + 1),
           *yv = dalloc(mr);
    if (!V || !Z) { free(V); free(Z); free(w); free(fs); free(t); free(H); free(cs); free(sn); free(g); free(yv); return ORC_ERR_MEM; }
    /* scaled: solve diag(A)^{-1} A u = diag(A)^{-1} f; the preconditioner of
     * that system is M^{-1} diag(A). */
    for (size_t k = 0; k < n; k++) fs[k] = scaled ? f[k] / aC[k] : f[k];
    double fn = nrm2(n, fs);
    double target = tol_abs ? tol : tol * fn;
    int it = 0, status = ORC_ERR_NOCONV, maxcyc = 0;
    double res = 0.0;
    for (;;) {
        sys_apply(N, aW, aE, aS, aN, aC, u, w, transpose, scaled);
        for (size_t k = 0; k < n; k++) w[k] = fs[k] - w[k];
        double beta = nrm2(n, w);
        res = beta;
        if (beta <= target || fn == 0.0) { status = ORC_OK; break; }
        if (it >= maxit) break;
        for (size_t k = 0; k < n; k++) V[k] = w[k] / beta;
        for (int i = 0; i <= mr; i++) g[i] = 0.0;
        g[0] = beta;
        int j, kdim = 0;
        for (j = 0; j < mr && it < maxit; j++) {
            double *vj = V + n * j, *zj = Z + n * j;
            if (P) {
                const double *src = vj;
                if (scaled) { for (size_t k = 0; k < n; k++) t[k] = vj[k] * aC[k]; src = t; }
                int c = orc_prec_apply(P, src, zj, transpose);
                if (c > maxcyc) maxcyc = c;
            } else memcpy(zj, vj, n * sizeof(double));
            sys_apply(N, aW, aE, aS, aN, aC, zj, w, transpose, scaled);
            for (int i = 0; i <= j; i++) {
                double *vi = V + n * i, h = 0.0;
                for (size_t k = 0; k < n; k++) h += w[k] * vi[k];
                H[(size_t)i * mr + j] = h;
                for (size_t k = 0; k < n; k++) w[k] -= h * vi[k];
            }
            double hn = nrm2(n, w);
            H[(size_t)(j + 1) * mr + j] = hn;
            if (hn != 0.0) for (size_t k = 0; k < n; k++) V[n * (j + 1) + k] = w[k] / hn;
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * mr + j], b = H[(size_t)(i + 1) * mr + j];
                H[(size_t)i * mr + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * mr + j] = -sn[i] * a + cs[i] * b;
            }
            double a = H[(size_t)j * mr + j], b = H[(size_t)(j + 1) * mr + j];
            double d = sqrt(a * a + b * b);
            cs[j] = d == 0.0 ? 1.0 : a / d;
            sn[j] = d == 0.0 ? 0.0 : b / d;
            H[(size_t)j * mr + j] = d;
            H[(size_t)(j + 1) * mr + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            it++;
            kdim = j + 1;
            if (fabs(g[j + 1]) <= target || hn == 0.0) break;
        }
        if (kdim == 0) break;
        for (int i = kdim - 1; i >= 0; i--) {
            double s = g[i];
            for (int k2 = i + 1; k2 < kdim; k2++) s -= H[(size_t)i * mr + k2] * yv[k2];
            yv[i] = s / H[(size_t)i * mr + i];
        }
        for (int i = 0; i < kdim; i++) {
            double *zi = Z + n * i;
            for (size_t k = 0; k < n; k++) u[k] += yv[i] * zi[k];
        }
    }
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = fn > 0 ? res / fn : 0.0;
    if (max_cycles_out) *max_cycles_out = maxcyc;
    free(V); free(Z); free(w); free(fs); free(t); free(H); free(cs); free(sn); free(g); free(yv);
    return status;
}

/* ------------------------------------------------------------------------
 * Adjoint gradients.  With A(c1,c2,r) u = f and A^T lam = dJ/du:
 *   dJ/df = lam,  dJ/dtheta = -lam^T (dA/dtheta) u.
 * From the stencil of Sec. 3, row (i,j) of A u contains
 *   c1_ij (u_ij - u_{i+1,j}) / h_{i+1} + c2_ij (u_ij - u_{i,j+1}) / k_{j+1}
 *   + r_ij u_ij   (u = 0 on the boundary),
 * so g_c1 = -lam (u - u_E)/h_{i+1}, g_c2 = -lam (u - u_N)/k_{j+1},
 * g_r = -lam u.  The mesh is held fixed.
 * ---------------------------------------------------------------------- */
void orc_grad(int N, const double *x, const double *y, const double *u, const double *lam,
              double *g_c1, double *g_c2, double *g_r)
{
    int M = N - 1;
    for (int j = 1; j <= M; j++)
        for (int i = 1; i <= M; i++) {
            size_t k = ix(N, i, j);
            double uE = (i < M) ? u[k + 1] : 0.0;
            double uN = (j < M) ? u[k + M] : 0.0;
            g_c1[k] = -lam[k] * (u[k] - uE) / (x[i + 1] - x[i]);
            g_c2[k] = -lam[k] * (u[k] - uN) / (y[j + 1] - y[j]);
            g_r[k] = -lam[k] * u[k];
        }
}
