/*
 * pint.h -- C ABI of the GB300 (sm_103a) library for the vectorised
 * parallel-in-time block solve of
 *     Engwer, Schell & Dreier, "Vectorized Parallel in Time methods for
 *     low-order discretizations with application to Porous Media problems",
 *     arXiv 2504.02117.
 *
 * Problem (Sec. 1, Eq. problem):  M y'(t) + K y(t) = b(t), M diagonal here.
 * s coupled time steps / DIRK stages give the matrix equation of
 * Eq. general-system-time-steps / Eq. time-stepping-matrices-multiple-
 * parallel-time-steps, in residual form (Sec. 2.2, sign read as "+F A2^T"):
 *     R(Y) = M Y A1^T + (K Y - B) A2^T - B0,         Y, B, B0, R in R^{N x s}.
 * It is solved by the splitting of Eq. matrix-splitting and the fixed point of
 * Eq. matrix-fixed-point-equation, written as defect correction
 *     R = R(Y);  (alpha M + beta K) V = R  (block GMRES);  Y <- Y - V,
 * alpha = A1[0][0] (= 1/tau), beta = A2[0][0].
 *
 * Conventions
 *  - Every call returns an int status (PINT_OK = 0 or a PINT_ERR_* code);
 *    pint_last_error(ctx) returns a message for the last failing call.
 *  - Block vectors (Y, B, B0, R, ...) are N x s ROW-MAJOR float64 arrays: the
 *    s values of one row are contiguous (one row = the s "SIMD lanes" of
 *    Sec. 3, one per coupled step). Unless a call says otherwise they are
 *    DEVICE pointers, borrowed: the caller owns them and keeps them alive until
 *    the work enqueued on `stream` has completed. A NULL B or B0 means zero.
 *  - Small coupling matrices (A1, A2, tableaux) are HOST row-major arrays,
 *    copied by the call.
 *  - Handles are opaque and owned by the library; free them with the matching
 *    *_destroy call. A context serves one device; calls on the same handle
 *    must not run concurrently from several host threads.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it. Calls documented "synchronous" wait for
 *    their own work on that stream before returning (they read convergence
 *    words on the host).
 *  - Device memory is accounted against the context's hbm_budget; a call that
 *    would exceed it fails with PINT_ERR_NOMEM before launching anything.
 */
#ifndef PINT_H
#define PINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  PINT_OK = 0,
  PINT_ERR_INVALID = 1,       /* bad argument (size, NULL, s out of range) */
  PINT_ERR_NOMEM = 2,         /* budget or cudaMalloc exhausted             */
  PINT_ERR_CUDA = 3,          /* a CUDA runtime call failed                 */
  PINT_ERR_NOT_CONVERGED = 4, /* iteration limit reached; stats are filled  */
  PINT_ERR_BREAKDOWN = 5,     /* NaN/Inf met in a residual or factorisation */
  PINT_ERR_TIMEOUT = 6        /* a device-side wait exceeded its time limit */
};

#define PINT_MAX_S 16         /* maximum block width s                      */
#define PINT_MAX_RESTART 64   /* maximum GMRES restart length               */

enum { PINT_MEM_HOST = 0, PINT_MEM_DEVICE = 1 };
enum { PINT_PC_NONE = 0, PINT_PC_JACOBI = 1, PINT_PC_ILU0 = 2 };
/* Arithmetic of the inner block GMRES. Outer residuals, updates, column norms
 * and the s x s / Hessenberg factorisations are always float64. */
enum {
  PINT_FP64 = 0,   /* matrix, vectors, Gram products in float64               */
  PINT_FP32 = 1,   /* float32 matrix + vectors, float32 products, float64
                      cross-block Gram reduction; float64 refinement outside */
  PINT_BF16 = 2    /* as PINT_FP32 but the SpMM matrix values are bfloat16    */
};

enum { PINT_SOLVER_GMRES = 0, PINT_SOLVER_CG = 1, PINT_SOLVER_BICGSTAB = 2,
       PINT_SOLVER_GLOBAL = 3 };

typedef struct pint_ctx_s* pint_ctx;
typedef struct pint_op_s* pint_op;
typedef struct pint_problem_s* pint_problem;
typedef struct pint_batch_plan_s* pint_batch_plan;

typedef struct {
  double tol;        /* outer: ||R_k||_2 <= tol ||F_k||_2, F = B A2^T + B0   */
  double inner_tol;  /* inner block GMRES: per-column relative reduction    */
  double max_step;   /* Newton calls only: if > 0, column k of the update V
                        is scaled by min(1, max_step / max_r |V_rk|) (a step
                        bound; the paper gives no globalisation). 0 = off    */
  double lscheme_L;  /* Richards Newton calls only: 0 = Newton, J = alpha
                        theta'(Y_0) + beta Df(t_0, Y_0). Otherwise the
                        L-scheme of Sec. 4.3: theta' is replaced by the
                        constant L and the conductivities are frozen at Y_0
                        (no derivative of kr): J = alpha L I + beta A(Y_0).
                        L > 0 is used as given; L < 0 takes the Lipschitz
                        constant of theta (pint_vg_lipschitz)                */
  int restart;       /* GMRES restart length m, 1..PINT_MAX_RESTART (30)    */
  int max_outer;     /* outer (defect-correction / Newton) iteration limit  */
  int max_inner;     /* block Arnoldi steps per inner solve                 */
  int precond;       /* PINT_PC_*                                           */
  int precision;     /* PINT_FP64 / PINT_FP32 / PINT_BF16                   */
  int solver;        /* inner solver: PINT_SOLVER_GMRES (block GMRES(restart),
                        right preconditioning), PINT_SOLVER_CG (breakdown-
                        free block CG, the paper's solver for symmetric
                        systems: J and the preconditioner must be symmetric
                        positive definite; uses 4 basis blocks, restart >= 3)
                        or PINT_SOLVER_BICGSTAB (block BiCGStab, the paper's
                        solver for the nonsymmetric linear problem, Sec. 4.1:
                        right preconditioning, the right-hand side block
                        deflated once by CholQR2; uses 9 basis blocks,
                        restart >= 8; a singular s x s system Rt^T V returns
                        PINT_ERR_BREAKDOWN). max_inner counts its iterations
                        (two operator and preconditioner applications each).
                        PINT_SOLVER_GLOBAL (pint_solve_block only, float64):
                        no splitting; global GMRES(restart) on the coupled
                        operator V -> M V A1^T + K V A2^T itself in the
                        Frobenius inner product, right-preconditioned column
                        by column with precond of J (the fixed point of
                        Eq. matrix-fixed-point-equation is not used; each
                        restart corrects Y from its true residual, inner_tol
                        is not used). Other values: PINT_ERR_INVALID         */
  int reserved[2];
} pint_opts;

typedef struct {
  int status;                   /* status of the call                        */
  int outer_its;                /* outer / Newton iterations                 */
  int inner_its;                /* block Arnoldi steps, all inner solves     */
  int restarts;                 /* GMRES restart cycles                      */
  int deflations;               /* CholQR columns deflated                   */
  int kernel_launches;          /* kernels this call enqueued                */
  double setup_ms;              /* preconditioner set-up (host clock)        */
  double solve_ms;              /* whole call (host clock)                   */
  double col_relres[PINT_MAX_S];/* final ||R_k|| / ||F_k|| per column        */
  double flops;                 /* algorithmic float64 operations (FMA = 2)
                                   when the call counts them (the batched
                                   solver), else 0                           */
} pint_stats;

/* Fill `o` with the defaults: tol 1e-10, inner_tol 1e-2, restart 30,
 * max_outer 200, max_inner 3000, Jacobi, FP64. */
void pint_opts_default(pint_opts* o);

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device`. hbm_budget bounds the device
 * bytes the library allocates (0 = 90% of free memory). The environment
 * variable PINT_GRAM_FUSE=0, read here, makes the context's block GMRES run
 * the first update and the second Gram product of block CGS2 as two
 * launches where it would otherwise fuse them into one pass (float32 inner
 * solves with s <= 4; same arithmetic, same results; for comparison). */
int pint_create(pint_ctx* ctx, int device, size_t hbm_budget);
int pint_destroy(pint_ctx ctx);
const char* pint_last_error(pint_ctx ctx);
/* Device bytes currently held by the library in this context. */
size_t pint_bytes_in_use(pint_ctx ctx);

/* --------------------------------------------------------------- operator */
/* Assemble the operator pair (K, M) of Eq. problem. K: CSR with n rows,
 * int32 rowptr[n+1], colind[nnz] (column indices sorted in each row, the
 * diagonal present), float64 K_vals[nnz]; M_diag[n] (diagonal mass) or NULL
 * for M = I. mem_space says where the four arrays live. The library copies
 * them into its own formats (CSR + SELL-32 slices, float32 / bfloat16
 * copies). Synchronous. */
int pint_operator_assemble(pint_ctx ctx, pint_op* op, int64_t n,
                           const int32_t* rowptr, const int32_t* colind,
                           const double* K_vals, const double* M_diag,
                           int mem_space, void* stream);
/* Same pattern, new values (e.g. a new Jacobian, Algorithm 1). Either
 * pointer may be NULL to keep the old values. */
int pint_operator_update_values(pint_op op, const double* K_vals,
                                const double* M_diag, int mem_space,
                                void* stream);
int pint_operator_destroy(pint_op op);
int64_t pint_operator_nnz(pint_op op);

/* Cell-centred FV operator of -div(D grad u) + div(v u) on [0,1]^d with
 * nx*ny*nz cells (nz = 1: 2-D; h = 1/nx), natural x-fastest numbering,
 * homogeneous Dirichlet ghost faces, first-order upwind convection, M = I.
 * D[n] is the per-cell diffusion coefficient (mem_space). Assembled on the
 * device. Synchronous. */
int pint_fv_convdiff(pint_ctx ctx, pint_op* op, int nx, int ny, int nz,
                     const double* D, double vx, double vy, double vz,
                     int mem_space, void* stream);

/* --------------------------------------------------------------- coupling */
/* Set the s x s time-stepping matrices A1, A2 (host, row-major) of
 * Eq. general-system-time-steps. The splitting of Eq. matrix-splitting uses
 * alpha = A1[0][0] and beta = A2[0][0]; the inner operator is
 * J = alpha M + beta K. 1 <= s <= PINT_MAX_S. */
int pint_set_coupling(pint_op op, int s, const double* A1, const double* A2);

/* Build A1, A2 for `steps` consecutive steps of the m-stage stiffly accurate
 * DIRK tableau A (m x m, row-major host) with step tau,
 * Eq. time-stepping-matrices-multiple-parallel-time-steps; with
 * eliminate_first != 0 the explicit first stage (a_11 = 0) is removed as in
 * Sec. 2.1 and e[i] = a_{i+2,1} (m-1 values) is returned for the B0 terms
 * e_i (b^n - K y^n). A1, A2 must hold (steps*m')^2 doubles, m' = m or m-1;
 * *s_out = steps*m'. */
int pint_coupling_from_dirk(const double* A, int m, int steps, double tau,
                            int eliminate_first, double* A1, double* A2,
                            double* e, int* s_out);

/* R = M Y A1^T + (K Y - B) A2^T - B0, all float64 N x s row-major (device).
 * One pass over K for all s columns; the s x s right-multiplies are applied
 * per row in registers (Sec. 3, BOP kernel, fused with the coupling). */
int pint_apply_coupled(pint_op op, const double* Y, const double* B,
                       const double* B0, double* R, void* stream);

/* Linear slab solve (Eq. matrix-fixed-point-equation as defect correction,
 * inner solves on J = alpha M + beta K by the block solver opts->solver:
 * block GMRES(m) by default, block BiCGStab or block CG; Jacobi or ILU(0)
 * preconditioning). Y: in = initial guess, out = solution. Stops when
 * every column satisfies ||R_k|| <= tol ||F_k|| (absolute tol if F_k = 0).
 * When A1 and A2 are lower triangular, a converged leading run of columns
 * stays converged (column k's residual depends on columns 0..k only): the
 * inner solves then take only the trailing columns (a power-of-two count
 * holding every unconverged one) and the leading ones are left as they are.
 * Synchronous. Returns PINT_ERR_NOT_CONVERGED (stats filled) at max_outer,
 * PINT_ERR_BREAKDOWN on a non-finite residual. */
int pint_solve_block(pint_op op, const double* B, const double* B0, double* Y,
                     const pint_opts* opts, pint_stats* stats, void* stream);

/* One slab solve of pint_solve_batch: Y solves M Y A1^T + (K Y - B) A2^T = B0
 * (Eq. general-system-time-steps) for the operator and coupling of `op`. */
typedef struct {
  pint_op op;          /* coupling set; several jobs may share one operator    */
  const double* B;     /* N x s row-major device, or NULL                      */
  const double* B0;    /* N x s row-major device, or NULL                      */
  double* Y;           /* N x s row-major device: in initial guess, out result;
                          the Y of different jobs must not overlap             */
} pint_batch_job;

/* Many slab solves (uneven N and s, each with its own operator and coupling)
 * in ONE persistent kernel launch: thread-block clusters of `cluster_ctas`
 * CTAs (1..16; 0 = pint_batch_auto_cluster) of `cta_threads` threads (128,
 * 256 or 512; 0 = pint_batch_auto_threads) take jobs from a device queue and
 * run each whole solve inside the cluster, with no host round trip per
 * Arnoldi step. The method per job is the one of PINT_SOLVER_GLOBAL in
 * pint_solve_block (global GMRES(opts->restart) on the unsplit coupled
 * operator, restarted as defect correction from the true residual, same
 * stopping test; modified Gram-Schmidt when a job runs on one CTA, two
 * classical passes on a cluster), float64, right preconditioned by Jacobi of
 * J = alpha M + beta K or by none: opts->precision must be PINT_FP64,
 * opts->precond PINT_PC_JACOBI or PINT_PC_NONE and opts->restart at most 32,
 * else PINT_ERR_INVALID. opts->solver and inner_tol are not used. A job's
 * result does not depend on the other jobs of the batch (fixed reduction
 * order for a given cluster size and CTA width). `stats`: NULL or njobs entries, filled per job (solve_ms is the whole
 * call). Device memory for (restart + 3) N s doubles per resident cluster is
 * taken from the context budget for the call. Synchronous. Returns PINT_OK
 * when every job converged, PINT_ERR_BREAKDOWN if any job met a non-finite
 * residual, else PINT_ERR_NOT_CONVERGED; per-job status is in stats. */
int pint_solve_batch(pint_ctx ctx, int njobs, const pint_batch_job* jobs,
                     const pint_opts* opts, int cluster_ctas, int cta_threads,
                     pint_stats* stats, void* stream);

/* Resident form of pint_solve_batch for repeated solves of the same jobs
 * (a serving loop, a bench): pint_batch_plan_create validates the jobs, copies
 * their couplings and descriptors to the device, allocates the workspace of
 * every resident cluster once and captures the launch (queue reset + the
 * persistent kernel) as a CUDA graph; it waits for its own copies on
 * `stream`. pint_batch_plan_run replays the graph on `stream`, waits for it
 * and fills `stats` (NULL or njobs entries); it returns as pint_solve_batch.
 * The caller writes new B, B0 and initial Y into the same device buffers
 * between runs. The plan borrows the operators and the job buffers: they must
 * stay alive and unchanged (no pint_set_coupling, pint_operator_update_values
 * or destroy) until pint_batch_plan_destroy, which waits for the device and
 * frees the plan's memory. */
int pint_batch_plan_create(pint_ctx ctx, int njobs, const pint_batch_job* jobs,
                           const pint_opts* opts, int cluster_ctas, int cta_threads,
                           pint_batch_plan* plan, void* stream);
int pint_batch_plan_run(pint_batch_plan plan, pint_stats* stats, void* stream);
/* The launch shape the plan took: CTAs per cluster, threads per CTA and the
 * number of clusters launched (resident at once, at most njobs). */
int pint_batch_plan_shape(pint_batch_plan plan, int* cluster_ctas, int* cta_threads,
                          int* resident_clusters);
int pint_batch_plan_destroy(pint_batch_plan plan);

/* The cluster size pint_solve_batch takes for cluster_ctas = 0: C doubles
 * from 1 (up to 16) while the largest job's N s / C exceeds the batch's total
 * N s per SM and the largest job keeps at least 256 rows per CTA. 0 when a
 * job has no operator or coupling. */
int pint_batch_auto_cluster(pint_ctx ctx, int njobs, const pint_batch_job* jobs);

/* The CTA width pint_solve_batch takes for cta_threads = 0 with clusters of
 * cluster_ctas CTAs: 256 for clusters of 16, else 512. */
int pint_batch_auto_threads(pint_ctx ctx, int njobs, int cluster_ctas);

/* shift((Y_1,...,Y_s)) = (Y_2,...,Y_s,Y_s) in place (Sec. 2.2, Eq. shift). */
int pint_shift(double* Y, int64_t n, int s, void* stream);

/* ------------------------------------------------ nonlinear problems (a11) */
enum { PINT_PROBLEM_DIFFREACT = 1, PINT_PROBLEM_RICHARDS = 2 };
/* Nonlinear FV problem M(y)' + f(t,y) = 0 on an nx*ny*nz grid.
 *  DIFFREACT: u_t = div((1+u^2) grad u) + u(1-u) + src(t), M = I, zero-flux
 *             boundary, moving-circle source of Sec. 4.2; params unused.
 *  RICHARDS:  d/dt theta(psi) - div(K_S kr(psi) grad(psi + z)) = 0 with the
 *             van Genuchten-Mualem relations (Eq. RelationshipsThetaK);
 *             params = {alpha, n, theta_r, theta_s, dt_D}; field = K_S[n]
 *             (device); top patch (x,y < 1/2) Dirichlet ramp -2 -> 0.2 over
 *             dt_D, other faces no-flow.
 * The problem builds its own operator (stencil pattern) reachable through
 * pint_problem_operator. */
int pint_problem_create(pint_ctx ctx, pint_problem* prob, int kind, int nx,
                        int ny, int nz, const double* params,
                        const double* field, void* stream);
int pint_problem_destroy(pint_problem prob);
/* Lipschitz constant of the van Genuchten theta(psi) for params = {alpha, n,
 * theta_r, theta_s}: sup theta' = (theta_s - theta_r) m n alpha x^(n-1)
 * (1 + x^n)^(-m-1) at x^n = m, m = 1 - 1/n (the L of the L-scheme, Sec. 4.3).
 * Host only; PINT_ERR_INVALID for n <= 1, alpha <= 0 or theta_s <= theta_r. */
int pint_vg_lipschitz(const double* params, double* L);
pint_op pint_problem_operator(pint_problem prob);
/* mass_out = M(y), f_out = f(t, y) for one column y[n] (either output may
 * be NULL). */
int pint_problem_eval(pint_problem prob, double t, const double* y,
                      double* mass_out, double* f_out, void* stream);
/* R = M(Y) A1^T + F(T, Y) A2^T - B0 with the coupling of the problem's
 * operator, times[s] (host) the stage times (Eq. matrix-equation-pipelining
 * residual, sign read as "+F A2^T"). */
int pint_problem_residual(pint_problem prob, const double* times,
                          const double* Y, const double* B0, double* R,
                          void* stream);
/* One simplified-Newton iteration of Algorithm 1 on the current window:
 * R = R(Y); if ||R_0|| <= tol * ||B0_0|| (tol alone if B0_0 = 0) set
 * *converged = 1 and
 * return; else J = alpha M'(Y_0) + beta Df(t_0, Y_0) (or the L-scheme matrix
 * when opts.lscheme_L != 0), solve J V = R with block GMRES (inner_tol),
 * Y <- Y - V (each column's step bounded by opts.max_step when it is > 0),
 * *converged = 0. Synchronous. */
int pint_newton_step(pint_problem prob, const double* times, double* Y,
                     const double* B0, const pint_opts* opts, int* converged,
                     pint_stats* stats, void* stream);
/* Algorithm 1 ("Block Krylov Time Stepping with Pipelining"): windows of s
 * consecutive stages of the stiffly accurate DIRK tableau (A, c) (m stages,
 * host arrays) starting from Y = (y0, ..., y0), shifted by one stage whenever
 * column 0 has converged, for `nstages` global stages. stages_out is N x
 * nstages ROW-MAJOR (device): column g = converged stage g. Synchronous. */
int pint_pipeline_run(pint_problem prob, const double* A, const double* c,
                      int m, double tau, int s, const double* y0,
                      int nstages, double* stages_out, const pint_opts* opts,
                      pint_stats* stats, void* stream);

/* --------------------------------------------------------------- profiler
 * Kernel families, for per-family CUDA-event timing. When the profiler is on,
 * each family's launches are bracketed by events on the launching stream;
 * every launch also books the family's algorithmic bytes and flops (the
 * CSR-form figures: matrix values + int32 column indices + rowptr, each
 * block vector read once and written once). */
enum {
  PINT_K_COUPLED = 0, /* fused coupled residual (linear and nonlinear)        */
  PINT_K_SPMM,        /* inner operator apply J X                             */
  PINT_K_GRAM,        /* block Gram products [V]^T W                          */
  PINT_K_UPDATE,      /* block AXPY with a small matrix                       */
  PINT_K_CHOLQR,      /* CholQR2 (its Gram, Cholesky, scaling)                */
  PINT_K_HESS,        /* block Hessenberg least squares                       */
  PINT_K_ILU,         /* ILU(0) factorisation and sweeps                      */
  PINT_K_NORM,        /* column norms                                         */
  PINT_K_VEC,         /* outer update, casts, axpy, shift, B0 terms           */
  PINT_K_NL,          /* nonlinear pointwise, Jacobian and single-column eval */
  PINT_K_COUNT
};
/* Profiler flags: bit 0 = CUDA-event timing per kernel family, bit 1 = an
 * NVTX range named after the family ("coupled", "spmm", "gram", "update",
 * "cholqr", "hess", "ilu", "norm", "vec", "nl") around each of its launches
 * (for ncu --nvtx filtering; free when no tool is attached). 0 turns both
 * off. Launch, byte and flop counts are always kept. Values outside 0..3:
 * PINT_ERR_INVALID. */
int pint_profile_enable(pint_ctx ctx, int on);

/* Per-column residual history of the last pint_solve_block (one row per
 * outer iteration: ||R_k|| / ||F_k||, k = 0..s-1, the quantity the paper
 * plots per step in Sec. 4) or pint_pipeline_run (one row per Newton /
 * L-scheme iteration of the window); pint_newton_step appends a row per
 * call. `out` (host, may be NULL) receives min(rows, max_rows) rows of s
 * doubles, row-major; *rows and *s (may be NULL) the recorded row count
 * and width. Up to 4 Mi values are kept. The batched solver keeps none. */
int pint_residual_history(pint_ctx ctx, double* out, int max_rows, int* rows, int* s);
int pint_residual_history_reset(pint_ctx ctx);

/* Checked build (libpint_bounds.so, -DPINT_BOUNDS): every matrix column
 * index a kernel gathers through (the coupled residual, the SELL SpMM, the
 * batched solver's operator rows) is checked against the row count before
 * use; a bad index is counted, the first is recorded and its access is
 * skipped. pint_bounds_report waits for the device and returns, since the
 * last report, the count and the first record (site 1 coupled residual, 2
 * SELL SpMM, 3 batched operator rows, 99 pint_test_bounds; the index and its
 * bound), then clears them. In the normal build *count = -1. Any output
 * pointer may be NULL. */
int pint_bounds_report(pint_ctx ctx, long long* count, int* site, long long* index,
                       long long* bound);
/* Test entry of the checked build: evaluates one check of `index` against
 * `bound` on the device (site 99). Nothing is accessed through the index in
 * either build; in the checked build a failing check is recorded. */
int pint_test_bounds(pint_ctx ctx, long long index, long long bound);
/* Synchronizes the device, folds finished event pairs into the totals and
 * returns family `k`'s totals since the last reset (any pointer may be
 * NULL). */
int pint_profile_read(pint_ctx ctx, int k, double* ms, double* bytes,
                      double* flops, long long* launches);
int pint_profile_reset(pint_ctx ctx);
/* Kernels this context has launched since it was created. */
long long pint_kernel_launches(pint_ctx ctx);

/* ------------------------------------------- building blocks (test access)
 * The kernels of the inner solve, exposed for parity tests. `precision`
 * selects float64 (PINT_FP64: double arrays) or float32 (PINT_FP32: float
 * arrays); H, R and norms are always float64. V holds nb blocks of N x s
 * row-major each, block b at V + b*n*s. */
/* Z = J X with J = alpha M + beta K of the current coupling (float64). */
int pint_inner_apply(pint_op op, const double* X, double* Z, void* stream);
/* Z = J X with the float32 (PINT_FP32) or bfloat16 (PINT_BF16) copy of J
 * that the low-precision inner solves use; X, Z float32 N x s (device, must
 * not alias), float32 accumulation. Asynchronous. */
int pint_inner_apply_lowp(pint_op op, int precision, const float* X, float* Z,
                          void* stream);
/* Z = P^{-1} X for the preconditioner of `precond` (float64), set up from
 * J on first use. */
int pint_precond_apply(pint_op op, int precond, const double* X, double* Z,
                       void* stream);
/* Z = P^{-1} X with the float32 copy of the ILU(0) factors that the float32
 * and bf16 inner solves use (X, Z: float32 N x s, device, must not alias).
 * Factors J on first use like pint_precond_apply. */
int pint_ilu0_apply_f32(pint_op op, const float* X, float* Z, void* stream);
/* H[(b*s+i)*s + k] = sum_r V_b[r][i] W[r][k]  ((nb*s) x s, float64, device).
 * nb*s <= 1024. Synchronous: it reads the device error word of the bulk-copy
 * pipeline afterwards (PINT_ERR_TIMEOUT when one of its waits ran out). */
int pint_block_gram(pint_ctx ctx, int precision, int64_t n, int s, int nb,
                    const void* V, const void* W, double* H, void* stream);
/* W[r][k] -= sum_{b,i} V_b[r][i] H[(b*s+i)*s + k]. */
int pint_block_update(pint_ctx ctx, int precision, int64_t n, int s, int nb,
                      const void* V, const double* H, void* W, void* stream);
/* CholQR2: W <- Q, R (s x s, device, row-major upper) with W_in = Q R;
 * deflated columns of Q are zero. */
int pint_cholqr2(pint_ctx ctx, int precision, int64_t n, int s, void* W,
                 double* R, void* stream);
/* Same product as pint_block_gram, for callers that cannot allocate device
 * memory: pint_block_gram needs a context, and creating one calls cudaMalloc.
 * Frameworks whose caching allocator owns the whole device pool, real-time
 * loops that must never allocate, and code that must not take the implicit
 * synchronisation of cudaMalloc/cudaFree can call this one instead. The paper
 * has no counterpart; it is an interface convenience.
 *  - No context; no cudaMalloc, cudaFree or other allocating call. The
 *    cross-CTA partial sums live in a fixed 4 MiB float64 array in the
 *    library's device memory, held on every device that loads the library
 *    until the process exits.
 *  - Limits: nb * s * s <= 4096 (the scratch) and nb * s <= 1024 (basis
 *    columns one Gram CTA covers); otherwise PINT_ERR_INVALID with a message
 *    from pint_last_error(NULL). 1 <= s <= 16; V, W 16-byte aligned.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address and keeps it for the life of the process; make
 *    that first call before any stream capture. A cudaDeviceReset of that
 *    device invalidates the kept address: do not call this entry point on a
 *    device after resetting it.
 *  - All calls share the array, which keeps the last call's contents; every
 *    call overwrites the part it reads. Calls that overlap on the GPU (other
 *    streams, other host threads) race on it and must be serialised by the
 *    caller.
 * Runs on the current device and `stream`; asynchronous. */
int pint_block_gram_noalloc(int precision, int64_t n, int s, int nb,
                            const void* V, const void* W, double* H,
                            void* stream);
/* Test access to the bounded device waits (no paper counterpart). which = 0:
 * one thread waits, through the same bounded wait as the ILU(0) sweeps, for a
 * device flag that nothing sets; which = 1: one CTA waits, through the same
 * bounded mbarrier wait as the Gram kernel's bulk-copy ring, for a
 * transaction count that no copy delivers. The deadline is limit_ms
 * (0 < limit_ms <= 1000) after the wait starts; the wait then gives up,
 * raises its error word and the kernel returns (no trap, no copy in flight),
 * so the context stays usable. Synchronous. Returns PINT_ERR_TIMEOUT when
 * the wait ran out, as it must. */
int pint_test_wait_timeout(pint_ctx ctx, int which, double limit_ms, void* stream);
/* Measured float64 FMA throughput of the context's device (no paper
 * counterpart; the roofline denominator of the float64 kernels): eight
 * independent FMA chains per thread on 8 blocks of 256 threads per SM, best
 * of three CUDA-event-timed launches after a warm-up, 2 flops per FMA.
 * *tflops receives TFLOP/s. Synchronous; runs on the legacy default stream. */
int pint_fp64_fma_peak(pint_ctx ctx, double* tflops);
/* norms[k] = ||X_k||_2 (host array of s doubles). Synchronous. */
int pint_colnorms(pint_ctx ctx, int precision, int64_t n, int s,
                  const void* X, double* norms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PINT_H */
