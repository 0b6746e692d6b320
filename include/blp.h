/*
 * blp.h -- C ABI of the GB300 boundary-layer-preconditioned solver.
 *
 * Solves the upwind finite-difference discretisation of
 *     -eps * Lap(u) - c . grad(u) + r u = f   on (0,1)^2,  u = 0 on the boundary
 * (MacLachlan, Madden & Nhan, arXiv 2108.13468, eq. (2D) and the 5-point
 * stencil of Sec. 3) on a tensor-product Shishkin mesh (Sec. 3, eq. (tau
 * exponential)), by restarted flexible GMRES (Sec. 3.3) right-preconditioned
 * with the block-upper-triangular boundary-layer preconditioner of Sec. 3.1,
 * eq. (2D blocks), whose corner block is approximated by the multigrid
 * iteration of Sec. 3.2.
 *
 * Conventions shared by every call:
 *  - N is the number of mesh intervals per axis (even, 8 <= N <= 16384).
 *    Grid functions live on the (N-1)^2 interior nodes (x_i, y_j),
 *    1 <= i, j <= N-1, stored x-fastest: index (j-1)*(N-1) + (i-1), double.
 *  - Array arguments may be host or device (CUDA) pointers; the library
 *    queries the pointer kind and stages host arrays through its own device
 *    buffers.  The caller keeps ownership of every array it passes; the
 *    library never frees or retains caller pointers after a call returns.
 *  - All calls return an int status (BLP_OK = 0 on success, BLP_ERR_* on
 *    failure); nothing is thrown across the ABI.  On error the output arrays
 *    hold the best values computed so far (documented per call).
 *  - Work is issued on the stream set with blp_set_stream (default: the
 *    legacy default stream); calls return after the work has completed.
 *  - A handle is not thread safe; use one handle per host thread.
 */
#ifndef BLP_H
#define BLP_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BLP_OK 0
#define BLP_ERR_ARG 1      /* invalid argument (N odd or out of range, eps not in (0,1], null pointer, ...) */
#define BLP_ERR_COEF 2     /* coefficients violate the assumptions of Sec. 3: c1 < beta_x, c2 < beta_y, r < 0, or non-finite */
#define BLP_ERR_NOCONV 3   /* iteration limit reached before the tolerance */
#define BLP_ERR_TIMEOUT 4  /* a bounded device-side wait gave up (the kernel recorded it and returned) */
#define BLP_ERR_CUDA 5     /* a CUDA runtime call failed */
#define BLP_ERR_MEM 6      /* device or host allocation failed */

/* precision of the solve */
#define BLP_FP64 0   /* everything in double precision */
#define BLP_MIXED 1  /* FP32 preconditioner (all block sweeps and the corner multigrid) inside FP64 FGMRES */

/* stopping rules */
#define BLP_STOP_SCALED 0   /* ||D^-1 (f - A u)||_2 <= tol ||D^-1 f||_2, D = diag(A) (default) */
#define BLP_STOP_REL2 1     /* ||f - A u||_2 <= tol ||f||_2 (unscaled; FP64 floor may exceed tol for tiny eps) */
#define BLP_STOP_ABS2 2     /* ||f - A u||_2 <= tol (tol = 10 ln(N)/N reproduces the paper's rule, Sec. 3.3) */

typedef struct blp_handle blp_handle;

/* Problem and solver parameters.  Call blp_params_default first. */
typedef struct {
    double eps;                /* perturbation parameter, 0 < eps <= 1 */
    int N;                     /* intervals per axis */
    double sigma;              /* transition-point factor: tau = min(1/2, sigma*eps*ln(N)/beta) (default 2) */
    double beta_x, beta_y;     /* lower bounds of c1, c2 (default 1, 1) */
    int restart;               /* FGMRES restart length m (default 30) */
    int maxit;                 /* total FGMRES iteration limit (default 20000) */
    int precision;             /* BLP_FP64 or BLP_MIXED */
    int stop_mode;             /* BLP_STOP_* */
    double corner_reduction;   /* corner multigrid residual reduction factor (default 1e3, Sec. 3.2) */
    int corner_max_cycles;     /* cap on corner cycles per application (default 50) */
    int corner_fixed_cycles;   /* >0: exactly this many corner cycles (M becomes a fixed linear map) */
    int check_coefficients;    /* nonzero: blp_setup validates c1, c2, r (default 1) */
    int mesh;                  /* BLP_MESH_SHISHKIN (default), BLP_MESH_GRADED or BLP_MESH_PARABOLIC */
    int layer_intervals;       /* NL: intervals on [0,tau] per axis, 0 (default) = N/2; other values
                                  give the general Shishkin mesh of blp_mesh_q (BLP_MESH_SHISHKIN only) */
    int device_driven;         /* 1: run the restarted FGMRES of a solve (Sec. 3.3) as one CUDA graph whose
                                  conditional nodes take every restart, iteration and corner-cycle decision
                                  on the device: the same kernels and results as the host-driven loop, bit
                                  for bit, with one host synchronisation per solve instead of two or three
                                  per iteration.  Applies to the scaled stopping rule on a capturable
                                  stream; the graph is built at the handle's first solve of each precision
                                  and direction and replayed afterwards.  0 (default): the host drives the
                                  loop (measured faster on GB300, see the design notes).  The environment
                                  variable BLP_SOLVE_GRAPH=0/1 overrides it at blp_setup. */
} blp_params;

#define BLP_MESH_SHISHKIN 0    /* piecewise-uniform layer mesh (blp_mesh) */
#define BLP_MESH_GRADED 1      /* graded layer mesh, same tau and split (blp_mesh_graded) */
/* One parabolic and one exponential layer (Sec. 3, eq. (tau parabolic);
 * Sec. 3.2, first case): blp_mesh in x (beta_x = C_low), blp_mesh_parabolic
 * in y (beta_y is not used; c2 >= 0 is required instead of c2 >= beta_y), the
 * blocks M_II, M_YY, M_XX of Sec. 3.1 unchanged, and the corner block
 * approximated by the semicoarsening cycle of Sec. 3.2: rows rescaled by
 * hb_i kb_j, coarsening by 2 in x only, operator-induced interpolation from
 * the North-South collapsed stencil, restriction P^T, Galerkin (nine-point)
 * coarse operators, downstream point Gauss-Seidel, V(1,1), four coarsest
 * sweeps, cycles until the scaled corner residual falls by corner_reduction
 * (the paper takes 1e2 for this case).  Forward solves and forward
 * preconditioner applications only: blp_solve_adjoint and transposed
 * applications return BLP_ERR_ARG on such a handle. */
#define BLP_MESH_PARABOLIC 2

/* Statistics of the last solve. */
typedef struct {
    int status;             /* same as the return value */
    int iters;              /* FGMRES iterations */
    int restarts;           /* FGMRES restart cycles */
    int corner_cycles_max;  /* largest corner multigrid cycle count in any preconditioner application */
    double relres;          /* final relative residual in the stop_mode's norm (FP64, true residual) */
    double relres_unscaled; /* ||f - A u||_2 / ||f||_2 (FP64) */
    double t_solve_ms;      /* wall time of the solve call */
    double t_setup_ms;      /* wall time of blp_setup for this handle */
    int device_driven;      /* 1: the iteration ran as one CUDA graph (blp_params.device_driven);
                               0: the host drove the loop */
} blp_info;

/* Fill *p with defaults: eps = 1e-4, N = 128, sigma = 2, beta = 1, restart
 * 30, maxit 20000, FP64, scaled stopping, corner_reduction 1e3, 50 max
 * cycles, no fixed cycles, coefficient checks on, Shishkin mesh with N/2
 * layer intervals, host-driven iteration. */
void blp_params_default(blp_params *p);

/* S0. Shishkin mesh nodes (Sec. 2.2 eq. (tau 1D), Sec. 3 eq. (tau exponential)):
 * tau = min(1/2, sigma*eps*ln(N)/beta), N/2 equal intervals on [0,tau] and
 * on [tau,1]; x_i = (i/(N/2)) tau for i <= N/2, tau + ((i-N/2)/(N/2))(1-tau)
 * above, x_N = 1.  x: host array of N+1 doubles (caller-owned).  Returns tau,
 * or a negative value for invalid arguments. */
double blp_mesh(int N, double eps, double sigma, double beta, double *x);

/* Graded layer mesh (the Remark after Theorem (big bound): the analysis also
 * covers graded layer meshes such as Bakhvalov's).  This is the
 * Bakhvalov-Shishkin mesh: the same tau and N/2 + N/2 split as blp_mesh, the
 * interior nodes of blp_mesh, and on the layer
 *     x_i = -(sigma eps / beta) ln(1 - 2 (1 - 1/N) i / N),  0 < i < N/2,
 * so that exp(-beta x / (sigma eps)) falls linearly in i; x_{N/2} = tau.
 * When tau is capped at 1/2 the mesh is uniform.  Arguments, ownership and
 * errors as blp_mesh.  The preconditioner's blocks and the corner multigrid
 * (coarse nodes at even fine indices, transfer weights 1/2 and 1/4) are
 * unchanged on this mesh. */
double blp_mesh_graded(int N, double eps, double sigma, double beta, double *x);

/* General Shishkin mesh (the Remark on general Shishkin meshes): a share
 * q = NL/N of the intervals in the layer, tau = min(q, sigma*eps*ln(N)/beta),
 * NL equal intervals on [0,tau] and N-NL on [tau,1]:
 *     x_i = (i/NL) tau for i <= NL,  x_i = tau + ((i-NL)/(N-NL)) (1-tau) above,
 * x_N = 1.  NL = N/2 gives blp_mesh.  With blp_params.layer_intervals = NL the
 * blocks of Sec. 3.1 split at layer index NL: C = nodes i, j <= NL, and so on
 * (the paper develops the preconditioner for any number of layer and
 * interior points).  1 <= NL <= N-2.  x: host array of N+1 doubles.
 * Returns tau, or a negative value for invalid arguments. */
double blp_mesh_q(int N, int NL, double eps, double sigma, double beta, double *x);

/* Parabolic-layer mesh (Sec. 3, eq. (tau parabolic)), the y mesh of
 * BLP_MESH_PARABOLIC: tau = min(1/2, sigma sqrt(eps) ln(N)), N/2 equal
 * intervals on [0,tau] and on [tau,1], nodes by the rule of blp_mesh.
 * x: host array of N+1 doubles (caller-owned).  Returns tau, or a negative
 * value for invalid arguments. */
double blp_mesh_parabolic(int N, double eps, double sigma, double *x);

/* Assemble the operator (Sec. 3 stencil) and build the preconditioner
 * (Sec. 3.1 blocks, line factorisations, Sec. 3.2 corner hierarchy) on the
 * current CUDA device.  c1, c2, r: (N-1)^2 values at the interior nodes of
 * the mesh blp_mesh returns for (N, eps, sigma, beta_x) in x and beta_y in y.
 * On success *out owns all device memory of the solver; release it with
 * blp_destroy.  Errors: BLP_ERR_ARG, BLP_ERR_COEF (when check_coefficients),
 * BLP_ERR_MEM, BLP_ERR_CUDA; *out is NULL then. */
int blp_setup(const blp_params *p, const double *c1, const double *c2, const double *r, blp_handle **out);

/* Issue all further work of this handle on `stream` (a cudaStream_t). */
int blp_set_stream(blp_handle *h, void *stream);

/* Solve A u = f (Sec. 3.3 FGMRES with the Sec. 3.1 preconditioner).
 * f: right-hand side; u: initial guess on entry, solution on exit.
 * tol: tolerance for the handle's stop_mode.  info may be NULL.
 * BLP_ERR_NOCONV leaves the last iterate in u and its residual in info. */
int blp_solve(blp_handle *h, const double *f, double *u, double tol, blp_info *info);

/* Solve the adjoint system A^T lambda = g with the transposed preconditioner
 * M^T (block lower triangular, applied C, X, Y, I).  Same conventions as
 * blp_solve; lambda holds the initial guess on entry. */
int blp_solve_adjoint(blp_handle *h, const double *g, double *lambda, double tol, blp_info *info);

/* Adjoint gradient assembly for J(u(c1, c2, r, f)) with A u = f and
 * A^T lambda = dJ/du:  dJ/df = lambda,  dJ/dr = -lambda u,
 * dJ/dc1 = -lambda (u - u_E)/h_{i+1},  dJ/dc2 = -lambda (u - u_N)/k_{j+1}
 * (u_E, u_N the east/north neighbours, 0 on the boundary).  Any of the
 * three outputs may be NULL.  The mesh is held fixed. */
int blp_grad(blp_handle *h, const double *u, const double *lambda, double *g_c1, double *g_c2, double *g_r);

/* y = A u (transpose != 0: y = A^T u), unscaled operator, FP64. */
int blp_apply_operator(blp_handle *h, const double *u, double *y, int transpose);

/* One application of the preconditioner of the row-normalised system
 * D^-1 A (D = diag(A)): z = (D^-1 M)^-1 v = M^-1 D v, or with transpose != 0
 * z = (D^-1 M)^-T v.  precision: BLP_FP64 or BLP_MIXED (FP32 arithmetic).
 * *cycles (may be NULL) receives the corner multigrid cycle count. */
int blp_precond_apply(blp_handle *h, const double *v, double *z, int transpose, int precision, int *cycles);

/* One problem of a batch: its parameters, fields, right-hand side, initial
 * guess / solution, tolerance, and (on return) its statistics and status. */
typedef struct {
    blp_params params;             /* N, eps, precision, ... of this problem */
    const double *c1, *c2, *r;     /* (N-1)^2 fields, host or device */
    const double *f;               /* right-hand side */
    double *u;                     /* initial guess on entry, solution on exit */
    double tol;                    /* tolerance for params.stop_mode */
    blp_info info;                 /* out: statistics of this solve */
    int status;                    /* out: BLP_OK or the error of this problem */
} blp_batch_item;

/* Solve `count` independent problems (Sec. 3.3 solve of each; the batched
 * workload of many small problems with different N and eps).  Up to
 * `concurrency` problems (<= 0: 16) are in flight at once, each on its own
 * stream of the current device, set up, solved and released by one of
 * `concurrency` host threads.  Per-problem conventions are those of
 * blp_setup + blp_solve; items[i].status and items[i].info report each
 * problem.  Returns BLP_OK when every problem succeeded, else the status of
 * the first (lowest-index) failed problem; BLP_ERR_ARG for count < 0 or a
 * null array.  The caller's arrays must stay valid until the call returns. */
int blp_solve_batched(blp_batch_item *items, int count, int concurrency);

/* Launch settings of the downstream sweeps (the wavefront kernel of the
 * Sec. 3.1 interior solve and the Sec. 3.2 Gauss-Seidel smoother).  They
 * change the schedule of the sweeps, not what they compute: results agree
 * to rounding order under every setting.
 *   dts_chunk   rows of a strip's boundary column handed to the next strip at
 *               once: 8, 16 or 32, or 0 = by precision (32 FP32, 16 FP64);
 *               the launch falls back to a shorter chunk where the staging
 *               buffers would not fit in shared memory;
 *   dts_cluster CTAs per thread-block cluster, 1..16 (above 8: non-portable
 *               cluster sizes);
 *   two_step    bit 0: FP32 sweeps, bit 1: FP64 sweeps, use the recurrence
 *               substituted into itself once (two rows per three dependent
 *               FMAs) instead of one row per two;
 *   precond_ms  blp_autotune: measured device time of one preconditioner
 *               application with this setting; -1 when not tuned. */
typedef struct {
    int dts_chunk;
    int dts_cluster;
    int two_step;
    double precond_ms;
} blp_tuning;

/* Current setting of the handle (the defaults, or the BLP_DTS_CHUNK,
 * BLP_DTS_CLUSTER and BLP_DTS_TWO_STEP environment overrides read by
 * blp_setup, or the last blp_set_tuning / blp_autotune).  BLP_ERR_ARG for a
 * null argument. */
int blp_get_tuning(blp_handle *h, blp_tuning *t);

/* Use setting *t (precond_ms ignored) for the handle's later solves.
 * Replayed preconditioner graphs captured under another setting are
 * released (after the handle's stream has drained).  BLP_ERR_ARG for a
 * null argument or a value outside the ranges above. */
int blp_set_tuning(blp_handle *h, const blp_tuning *t);

/* Autotuner: times the preconditioner application in `precision`
 * (BLP_FP64 or BLP_MIXED) on this handle's problem, with a fixed
 * deterministic right-hand side, under every candidate setting (chunks 8,
 * 16, 32; cluster sizes 2 to 16 up to the widest block's strip count; one-
 * and two-step form for that precision), `reps` timed applications each
 * (<= 0: 3) after two warm-up ones, on the handle's stream with CUDA
 * events.  Keeps the fastest setting on the handle and writes it to *best
 * (may be NULL).  Allocates two vectors from the library's pool for the
 * duration.  BLP_ERR_ARG for a null handle or another precision; on a
 * CUDA or device error the handle's previous setting is restored and the
 * error returned. */
int blp_autotune(blp_handle *h, int precision, int reps, blp_tuning *best);

/* blp_solve_batched with autotuned launch settings: before the problems are
 * solved, each (N, precision) pair that this process has not tuned yet is
 * tuned once by blp_autotune on the first problem that has it (one at a
 * time, on a private stream); every problem then runs with the setting of
 * its pair.  The settings stay cached for later calls in the process.
 * Returns and reports as blp_solve_batched.  A pair whose tuning fails runs
 * with the default setting (each problem's own setup and solve report its
 * errors). */
int blp_solve_batched_tuned(blp_batch_item *items, int count, int concurrency);

/* One-dimensional method of Sec. 2, batched.  Problem k is
 *     -eps u'' - c(x) u' + r(x) u = f on (0,1),  u(0) = u(1) = 0     (eq. 1D),
 * discretised by the upwind scheme of eq. (stencil_1d) on the Shishkin mesh
 * of eq. (tau 1D) with tau = min(1/2, sigma eps ln(N) / c_low) and N/2
 * intervals on each side of tau, and solved by GMRES without restarts from
 * u = 0 on the left-preconditioned system M^-1 A u = M^-1 f, M of
 * eq. (block_M) (A on the layer block and both coupling entries, the upper
 * triangle of the interior block), the setting of Table 2, stopping at the
 * first iterate with ||f - A u||_inf <= stop (the rule of Sec. 2.5.1 with
 * K g(N) = stop), or after maxit iterations.
 *   N        intervals, even, 8 <= N <= BLP_1D_MAX_N
 *   c, r, f  DEVICE (or managed) arrays of N-1 values at the interior nodes
 *            x_1 .. x_{N-1} of that mesh (caller-owned, read only)
 *   u        DEVICE array of N-1 values: receives the last iterate
 *   maxit    1 .. BLP_1D_MAXIT
 *   iters, resid, status (out): iterations taken, ||f - A u||_inf of the
 *            returned u, BLP_OK or BLP_ERR_NOCONV (maxit reached) or
 *            BLP_ERR_ARG (this problem's arguments are invalid). */
#define BLP_1D_MAX_N 65536
#define BLP_1D_MAXIT 128
typedef struct {
    int N;
    double eps, c_low, sigma;
    const double *c, *r, *f;
    double *u;
    double stop;
    int maxit;
    int iters;
    double resid;
    int status;
} blp_1d_problem;

/* Solve `count` problems on `stream` (a cudaStream_t; NULL: the legacy
 * stream), one GPU thread per problem; returns after they have finished.
 * Workspace: (maxit + 10) (N - 1) + (maxit + 1) maxit doubles per problem,
 * allocated stream-ordered for the call.  Returns BLP_OK when every problem
 * met its stopping rule, else the status of the first problem that did not
 * (the others still run); BLP_ERR_ARG, with nothing launched, when count < 0,
 * probs is null or any problem's arguments are invalid (host pointers
 * included: they are refused, never dereferenced on the device); BLP_ERR_MEM
 * when the workspace cannot be allocated. */
int blp_solve_1d_batched(blp_1d_problem *probs, int count, void *stream);

/* Largest N accepted by blp_residual_noalloc (its fixed scratch holds four
 * partial sums per grid row: 4 * 8192 doubles = 256 KiB per device). */
#define BLP_NOALLOC_MAX_N 8192

/* Residual of the assembled operator without allocating anything and
 * without a handle.  The paper has no counterpart: this is a library
 * utility for callers that cannot allocate device memory when they check a
 * solution -- device memory already fully reserved, a path where the
 * device-wide synchronisation of cudaMalloc/cudaFree would stall other
 * streams, or a monitor that holds no blp_handle.
 *
 * Computes s = f - A u, with A the upwind 5-point operator that blp_setup
 * assembles for the tensor mesh x (N+1 nodes) by y (N+1 nodes), eps and the
 * fields c1, c2, r, and writes
 *     norms[0] = ||s||_2,        norms[1] = ||D^-1 s||_2,
 *     norms[2] = ||f||_2,        norms[3] = ||D^-1 f||_2     (D = diag(A)).
 * x, y, c1, c2, r, f, u: arrays in the current device's memory (or managed
 * memory), read only; fields have (N-1)^2 entries in the layout of the other
 * calls.  res: such an array of (N-1)^2 doubles receiving s, or NULL (the
 * norms are still computed).  norms: 4 doubles, host or device, or NULL.
 * stream: a cudaStream_t of the current device (NULL: legacy default
 * stream); the call returns after its work on that stream has completed.
 * Errors: BLP_ERR_ARG for N odd, N < 8, N > BLP_NOALLOC_MAX_N, eps outside
 * (0,1], or a null input array, a host array or another GPU's array;
 * BLP_ERR_CUDA when a CUDA call fails.
 * Memory: reduction partials live in one fixed device array per device
 * (BLP_NOALLOC_MAX_N bounds its size), held by every GPU that loads the
 * library until the process exits.  Each call looks up that array's device
 * address with the caller's device current.  The first call on a device also
 * loads this code onto the device, which is when the array is reserved: make
 * that first call during set-up, before device memory is fully reserved and
 * before any stream capture begins.  Every call on a device shares the array
 * and each call clears what must start at zero, so calls whose GPU work
 * overlaps (different streams, or several host threads) race: serialise
 * them. */
int blp_residual_noalloc(int N, const double *x, const double *y, double eps, const double *c1,
                         const double *c2, const double *r, const double *f, const double *u,
                         double *res, double *norms, void *stream);

/* Self-check of the device-side bounded waits (no counterpart in the
 * paper): one warp waits, with the same helpers the wavefront kernel uses
 * and a short iteration limit, for a shared-memory counter and an mbarrier
 * phase that nothing completes.  Both waits must give up and record a
 * timeout; the call returns BLP_ERR_TIMEOUT when they did (the expected
 * result), BLP_OK if either wait did not report, BLP_ERR_CUDA on a CUDA
 * failure.  The handle's error word is cleared afterwards, so the handle
 * stays usable. */
int blp_check_wait_timeout(blp_handle *h);

/* Release the handle and all its device memory.  NULL is ignored. */
void blp_destroy(blp_handle *h);

/* Static description of a status code. */
const char *blp_strerror(int status);

/* Number of kernels this handle has launched since blp_setup (a counter the
 * library keeps; used to report launch counts of timed regions). */
long long blp_kernel_launches(const blp_handle *h);

/* Optional per-kernel-class timing with CUDA events on the handle's stream.
 * blp_profile(h, 1) clears the counters and starts recording an event pair
 * around every launch; blp_profile(h, 0) stops.  blp_profile_read returns
 * the launch count, summed device time (ms) and summed algorithmic bytes
 * (the words each launch must read and write once, times the word size) of
 * class cls (0 <= cls < blp_kernel_class_count(); names from
 * blp_kernel_class_name).  Any output pointer may be NULL.  Recording adds
 * host overhead, so timed runs leave it off. */
int blp_profile(blp_handle *h, int enable);
int blp_profile_read(blp_handle *h, int cls, long long *count, double *total_ms, double *bytes);
/* Dependency-chain length of the recorded launches of class cls: the sum,
 * over its wavefront sweeps, of the steps a sweep cannot do in parallel
 * (mx + my - 1 anti-diagonals of a downstream Gauss-Seidel sweep).  Times a
 * step's latency it gives the latency floor the sweeps are measured against.
 * 0 for classes that are not wavefronts. */
int blp_profile_chain_steps(blp_handle *h, int cls, double *steps);
int blp_kernel_class_count(void);
const char *blp_kernel_class_name(int cls);

#ifdef __cplusplus
}
#endif
#endif
