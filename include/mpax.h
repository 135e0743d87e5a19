/*
 * mpax.h -- C ABI of the GB300 restarted-PDHG library (libmpax_gb300.so).
 *
 * The library solves problem (1) of the paper (Sec. 2),
 *
 *     min  1/2 x^T Q x + c^T x   s.t.   lc <= A x <= uc,   l <= x <= u,
 *
 * with r^2HPDHG (Algorithm 1; eqs. 3-4) when Q = 0 and rAPDHG (Algorithm 2;
 * eqs. 5-6) otherwise, after Ruiz and Pock-Chambolle diagonal scaling (Sec. 3).
 * Every step of the iteration runs in the library's own sm_103a kernels.
 *
 * Conventions for every entry point
 *   - Every call returns an mpax_status; it never aborts or exits.  On failure
 *     mpax_last_error() gives a message (thread-local; valid until the calling
 *     thread's next call into the library).
 *   - Vectors are dense, contiguous, FP64 unless the name says otherwise.
 *     Infinite bounds are IEEE +-INFINITY.
 *   - Sparse matrices are CSR: row_ptr (int64, rows+1 entries, row_ptr[0]=0,
 *     non-decreasing), col_idx (int32, strictly increasing within a row,
 *     0 <= col < cols), val (FP64).  nnz must be < 2^31.
 *   - `kind` says whether pointer arguments are host or device (CUDA) memory.
 *     Device pointers must belong to the current device.
 *   - `cuda_stream` is a cudaStream_t (may be NULL = the legacy default
 *     stream).  The library orders its work after the work already queued on
 *     that stream and makes that stream wait for the library's results, so a
 *     caller can treat every call as stream-ordered on `cuda_stream`.
 *   - Handles are not thread-safe; distinct handles are independent.
 */
#ifndef MPAX_H_
#define MPAX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mpax_status {
  MPAX_OK = 0,
  MPAX_ERR_INVALID_ARGUMENT = 1, /* bad sizes, unsorted CSR, NaN data, l > u ... */
  MPAX_ERR_CUDA = 2,             /* a CUDA runtime call failed                   */
  MPAX_ERR_OUT_OF_MEMORY = 3,    /* device allocation failed                     */
  MPAX_ERR_NOT_SOLVED = 4,       /* results requested before mpax_solve          */
  MPAX_ERR_DEVICE_TIMEOUT = 5,   /* a bounded device-side wait gave up           */
  MPAX_ERR_NUMERICAL = 6,        /* NaN/Inf appeared in the iterates             */
  MPAX_ERR_UNSUPPORTED = 7       /* option or input form the library does not take */
} mpax_status;

typedef enum mpax_mem_kind { MPAX_MEM_HOST = 0, MPAX_MEM_DEVICE = 1 } mpax_mem_kind;

/* Arithmetic of the iteration.  FP64: matrix, iterates and every vector in
 * FP64.  MIXED: scaled matrix, iterates and vectors stored and updated in
 * FP32 (SpMV accumulated in FP32); the KKT, duality-gap and restart
 * reductions, the step sizes and the primal weight stay FP64. */
typedef enum mpax_precision { MPAX_PREC_FP64 = 0, MPAX_PREC_MIXED = 1 } mpax_precision;

/* Outcome of a solve (optimal, infeasible, unbounded are the conclusive ones,
 * Sec. 4.5; the limits and numerical failure are not). */
typedef enum mpax_termination {
  MPAX_TERM_UNSOLVED = 0,
  MPAX_TERM_OPTIMAL = 1,
  MPAX_TERM_PRIMAL_INFEASIBLE = 2, /* LP: a Farkas dual ray was found (see below) */
  MPAX_TERM_DUAL_INFEASIBLE = 3,   /* LP: an unbounded primal ray was found */
  MPAX_TERM_ITERATION_LIMIT = 4,
  MPAX_TERM_TIME_LIMIT = 5,
  MPAX_TERM_NUMERICAL_ERROR = 6
} mpax_termination;

/* Solver options.  The first block follows the paper's Appendix A (defaults
 * there); the second block fixes the rules the paper names but does not state
 * (Sec. 3: step sizes, restarts, primal weight, scaling).  Always initialise
 * with mpax_options_default(). */
typedef struct mpax_options {
  int32_t verbose;            /* 0: print a line every display_frequency checks */
  int32_t display_frequency;  /* 10 */
  int32_t warm_start;         /* informational: x0/y0 of mpax_solve are used when non-NULL */
  int32_t feasibility_polishing; /* 0; 1: polish an OPTIMAL LP solve (eps_feas_polish);
                                    ignored for QPs */
  double eps_abs;             /* 1e-4 */
  double eps_rel;             /* 1e-4 */
  double eps_primal_infeasible; /* 1e-8.  LP infeasibility detection (Sec. 3): at each
                                   check the move since the restart cycle's anchor,
                                   (dx, dy), is tested.  Primal infeasible: y = dy on
                                   the recession cone of Y, lam = -A^T y, with
                                   ||lam - proj_Lambda(lam)|| <= eps * o and o > 0,
                                   o = sum lc y^+ - uc y^- + l lh^+ - u lh^- (finite
                                   terms, lh = proj_Lambda(lam)).  <= 0: off.  QPs are
                                   not tested. */
  double eps_dual_infeasible;   /* 1e-8.  Dual infeasible (unbounded LP): dx with
                                   ||(A dx, dx) - proj onto the recession cones of
                                   ([lc,uc], [l,u])|| <= eps * (-c^T dx), c^T dx < 0.
                                   <= 0: off.  In MIXED precision, where the FP32 rays
                                   cannot meet the tolerance, the stalled run continues
                                   in FP64 (see fp64_continuation), where the test is
                                   met. */
  double eps_feas_polish;       /* 1e-6.  With feasibility_polishing = 1, an LP solve
                                   that ends OPTIMAL is polished (Sec. 3.3) in FP64:
                                   the zero-objective problem from (x^, 0) until
                                   ||r_p|| <= eps (1 + ||b||), then the problem with
                                   every finite bound at zero from (0, y^) until
                                   ||r_d|| <= eps (1 + ||c||).  mpax_get_solution then
                                   returns that pair and mpax_stats its KKT values
                                   (optimality may relax: the gap is not re-tested). */
  int64_t iteration_limit;      /* INT64_MAX */
  double time_limit;            /* seconds, +inf */

  int32_t precision;          /* mpax_precision, FP64 */
  int32_t check_every;        /* 64: iterations between KKT/restart checks (1..1024) */
  int32_t ruiz_iters;         /* 10 */
  int32_t pock_chambolle;     /* 1: one Pock-Chambolle round, alpha = 1 */
  double reflection_gamma;    /* 1.0 (Algorithm 1); eq. 4 allows [0, 1] */
  double restart_sufficient;  /* 0.2 */
  double restart_necessary;   /* 0.8 */
  double restart_artificial;  /* 0.36 */
  double primal_weight_smoothing; /* 0.5 */
  double step_safety;         /* 0.998: eta = step_safety / ||A~||_2 */
  int32_t power_max_iter;     /* 1000.  0 (LPs, with pock_chambolle): no power
                                 iteration; ||A~||_2 := 1, the bound that the
                                 Pock-Chambolle round guarantees (Schur's test) */
  double power_tol;           /* 1e-4.  Power iteration for ||A~||_2 (and ||Q~||_2)
                                 from a fixed pseudo-random start vector (entries
                                 2u-1, u from SplitMix64 of the index); it stops
                                 when the last rise d of the estimate and the
                                 extrapolated remainder d q / (1 - q) (q: ratio of
                                 successive rises) are both <= power_tol times the
                                 estimate, which is then raised by the remainder */
  int32_t use_graphs;         /* 1: replay each check block as one CUDA graph */
  int32_t profile_kernels;    /* 0: 1 = time every fused SpMV launch with CUDA events
                                 (no graphs; for measurement only) */
  int32_t fp64_continuation;  /* 1: a MIXED solve whose relative KKT error stops
                                 improving (no 10% gain over max(stall_checks,
                                 checks so far / 4) checks) continues in FP64 from
                                 its FP32 point */
  int32_t stall_checks;       /* 8: the shortest stall window, in checks */
  int32_t record_tape;        /* 0.  1 (QP, FP64 precision): keep one record per check
                                 block -- step sizes, counters, restart flag and the
                                 block's start state (x, xavg, y, yavg), i.e.
                                 2(n + m) values -- for mpax_qp_unrolled_grad.  The
                                 records stay in device memory until the next
                                 mpax_solve or mpax_destroy. */
  int32_t spmv_kernel;        /* -1: autotuned.  Kernel of the A and A^T products of
                                 the iteration: 0 one warp per work item (at least
                                 20 CTAs of 2 warps per SM), 1 persistent warps with
                                 TMA-staged matrix rows, 2 as 0 with a register
                                 budget for 10 CTAs per SM.  All compute every
                                 product and sum in the same order, so results are
                                 identical bit for bit; -1 times each on the
                                 problem's own matrices, with the iteration's own
                                 half-step epilogues, at the first prepare (ten
                                 launches each) and keeps the fastest (another
                                 kind must beat 0 by 3%), cached for the process
                                 by matrix signature (rows, columns, nnz, LP or
                                 QP, precision, histogram of log2 row lengths) */
  int32_t batch_stage;        /* 1.  Ragged batch (mpax_batch_solve) with at most one
                                 instance per SM: an instance whose matrices, scaled
                                 data and iterates fit in 200 KB of shared memory is
                                 copied there whole and iterates without global-memory
                                 traffic.  0, or more instances than SMs: only each
                                 instance's two gathered vectors and row pointers are
                                 staged.  Results are identical bit for bit. */
} mpax_options;

typedef struct mpax_stats {
  int32_t termination;        /* mpax_termination */
  int32_t precision;
  int64_t iterations;         /* PDHG iterations taken */
  int64_t restarts;
  int64_t kkt_checks;
  double primal_obj, dual_obj, gap;  /* unscaled problem, at the returned point */
  double primal_res, dual_res;       /* ||r_p||_2, ||r_d||_2 */
  double rel_kkt;                    /* relative KKT error (see mpax_kkt) */
  double omega, eta, norm_A, norm_Q; /* final primal weight, eta, ||A~||, ||Q~|| */
  double prepare_seconds;            /* transpose + scaling + norms */
  double solve_seconds;              /* whole mpax_solve, host wall clock */
  int64_t kernel_launches;           /* library kernels launched by the last mpax_solve */
  /* profile_kernels = 1 only: summed CUDA-event milliseconds and launch counts of
   * [0] primal fused SpMV^T, [1] dual fused SpMV, [2] KKT SpMV, [3] KKT SpMV^T */
  double profile_ms[4];
  int64_t profile_launches[4];
  int64_t fp64_iterations;           /* iterations of the FP64 continuation (MIXED) */
  int64_t polish_iterations;         /* iterations of the two feasibility-polishing runs */
  int64_t backward_launches;         /* library kernels of the last mpax_qp_unrolled_grad */
  int32_t spmv_kernel[2];            /* kernel (mpax_options.spmv_kernel) of A, A^T */
  double spmv_tune_us[6];            /* autotuner timings of the last prepare that timed:
                                        A kinds 0, 1, 2, then A^T kinds 0, 1, 2
                                        (microseconds per launch; 0 = not timed) */
  /* profile_kernels = 1, QP only: the same for the product ahead of the primal
   * half-step (F~^T x_md for Q = D + F F^T, Q~ x_md for a general Q) */
  double profile_ms_aux;
  int64_t profile_launches_aux;
} mpax_stats;

typedef struct mpax_problem mpax_problem;

const char* mpax_version(void);
const char* mpax_last_error(void);
const char* mpax_status_string(mpax_status s);
void mpax_options_default(mpax_options* opts);

/* Create an LP: problem (1) with Q = 0 (Sec. 2).  m rows, n columns, CSR A.
 * All arrays are copied into library-owned device memory, so the caller may
 * free or reuse them when the call returns.  Validation: sizes >= 0,
 * CSR well formed and sorted, no NaN, l <= u, lc <= uc.  m = 0 or nnz = 0 is
 * allowed.  On success *out owns the problem (free with mpax_destroy). */
mpax_status mpax_lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                           const int32_t* col_idx, const double* val, const double* c,
                           const double* lc, const double* uc, const double* l,
                           const double* u, mpax_mem_kind kind, void* cuda_stream,
                           mpax_problem** out);

/* mpax_lp_create with FP32 values and vectors (row_ptr and col_idx as there).
 * They are widened to FP64 on entry, so the problem is exactly the FP64 problem
 * with those values; the iteration precision is still chosen by the options. */
mpax_status mpax_lp_create_f32(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                               const int32_t* col_idx, const float* val, const float* c,
                               const float* lc, const float* uc, const float* l,
                               const float* u, mpax_mem_kind kind, void* cuda_stream,
                               mpax_problem** out);

/* Create a convex QP with Q = diag(D) + F F^T (Sec. 2, eq. 1), D >= 0
 * (n entries), F an n x r CSR matrix (f_row_ptr has n+1 entries).  Other
 * arguments and ownership as mpax_lp_create. */
mpax_status mpax_qp_create_diag_lowrank(
    int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
    const double* val, const double* c, const double* lc, const double* uc, const double* l,
    const double* u, const double* D, int32_t r, int64_t f_nnz, const int64_t* f_row_ptr,
    const int32_t* f_col_idx, const double* f_val, mpax_mem_kind kind, void* cuda_stream,
    mpax_problem** out);

/* Problem (1) with a general sparse Q (Sec. 2, eq. 1): Q is n x n in CSR
 * (q_row_ptr n+1 int64 entries, q_col_idx sorted within each row, q_val),
 * symmetric positive semidefinite with BOTH triangles stored; symmetry and
 * definiteness are the caller's (not verified).  Q's diagonal joins the
 * column norms of the scaling, ||Q~||_2 comes from power iteration, and every
 * Q product of the iteration, the KKT test, the implicit adjoint and the
 * unrolled gradient is one SpMV with Q~ = D_c Q D_c.  Other arguments,
 * validation and ownership as mpax_lp_create.  In the differentiation calls the
 * gradient named dD is that of Q's diagonal. */
mpax_status mpax_qp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                           const int32_t* col_idx, const double* val, const double* c,
                           const double* lc, const double* uc, const double* l,
                           const double* u, int64_t q_nnz, const int64_t* q_row_ptr,
                           const int32_t* q_col_idx, const double* q_val, mpax_mem_kind kind,
                           void* cuda_stream, mpax_problem** out);

/* Solve from (x0, y0) given in the unscaled space (either may be NULL: zeros,
 * the paper's default start, Sec. 3.5).  Runs transpose, scaling, norm
 * estimation and the restarted iteration until the relative KKT test holds,
 * the iteration limit or the time limit is reached, or NaN appears (status
 * MPAX_ERR_NUMERICAL).  Returns after the device work is complete. */
mpax_status mpax_solve(mpax_problem* prob, const mpax_options* opts, const double* x0,
                       const double* y0, mpax_mem_kind kind);

/* Copy the returned point into caller-owned buffers: x (n), y (m) in the
 * unscaled space.  For LP that is the PDHG image (x^, y^) of the last
 * check (Algorithm 1); for QP the weighted averages (Algorithm 2).
 * Either pointer may be NULL.  MPAX_ERR_NOT_SOLVED before a solve. */
mpax_status mpax_get_solution(const mpax_problem* prob, double* x, double* y,
                              mpax_mem_kind kind);
mpax_status mpax_get_stats(const mpax_problem* prob, mpax_stats* stats);

/* Restarts of the last run (Algorithms 1/2; the restart rule and the primal-weight
 * update of Sec. 3 as mpax_options states them): *count receives how many there
 * were; the first min(*count, cap, 256) entries of iters / omega (HOST memory,
 * either nullable) receive the iteration count at which each restart happened
 * and the primal weight after its update.  For a MIXED solve continued in FP64
 * this is the FP64 run's log.  MPAX_ERR_NOT_SOLVED before a solve. */
mpax_status mpax_get_restart_history(const mpax_problem* prob, int32_t cap, int64_t* iters,
                                     double* omega, int32_t* count);

/* Free everything the handle owns.  NULL is a no-op. */
void mpax_destroy(mpax_problem* prob);

/* ---- Lower-level entry points (each step of the path on its own) ---------- */

/* Transpose, scaling and norm estimation for `opts` (what mpax_solve does
 * first).  Needed before the calls below. */
mpax_status mpax_prepare(mpax_problem* prob, const mpax_options* opts);

/* Scaling factors D_r (m), D_c (n) with A~ = diag(D_r) A diag(D_c), and
 * info[4] = {||A~||_2 estimate, ||Q~||_2 estimate, eta, omega_0}.  Any
 * pointer may be NULL. */
mpax_status mpax_get_scaling(const mpax_problem* prob, double* Dr, double* Dc, double* info,
                             mpax_mem_kind kind);

/* The device-built transpose of the (unscaled) A as CSR: rowptr_t (n+1),
 * col_t (nnz), val_t (nnz). */
mpax_status mpax_get_transpose(const mpax_problem* prob, int64_t* rowptr_t, int32_t* col_t,
                               double* val_t, mpax_mem_kind kind);

/* Set the iterate in the SCALED space.  LP: (x, y) = z^{n,k}, (x_aux, y_aux)
 * = the restart anchor z^{n,0}.  QP: (x, y) = current point, (x_aux, y_aux)
 * = the weighted averages.  k = inner counter, tau/sigma = step sizes. */
mpax_status mpax_set_iterate(mpax_problem* prob, const double* x, const double* y,
                             const double* x_aux, const double* y_aux, int64_t k, double tau,
                             double sigma, mpax_mem_kind kind);

/* Run `iters` plain iterations (no checks, no restarts) from the set iterate. */
mpax_status mpax_iterate(mpax_problem* prob, int64_t iters);

/* Read the iterate (SCALED space).  LP: (x, y) = z^{n,k} after the run,
 * (x_hat, y_hat) = the PDHG image of the last step.  QP: (x, y) current,
 * (x_hat, y_hat) = the weighted averages.  Any pointer may be NULL. */
mpax_status mpax_get_iterate(const mpax_problem* prob, double* x, double* y, double* x_hat,
                             double* y_hat, mpax_mem_kind kind);

/* Relative KKT quantities of the UNSCALED problem at (x, y) (unscaled); the
 * paper names them (primal feasibility, dual feasibility, duality gap; Sec. 3)
 * and this library evaluates them as
 *   r_p = A x - proj_[lc,uc](A x);   lam = Q x + c - A^T y;
 *   r_d = lam - proj_Lambda(lam), Lambda_j = R (both bounds finite), R+ (only
 *         l_j), R- (only u_j), {0} (neither);
 *   p = 1/2 x^T Q x + c^T x;
 *   d = -1/2 x^T Q x + sum(lc y^+ - uc y^-) + sum(l lh^+ - u lh^-), lh the
 *       projected lam, terms with an infinite bound dropped;
 *   rel = max(||r_p||/(1+||b||), ||r_d||/(1+||c||), |p-d|/(1+|p|+|d|)),
 *         b_i the finite one of (lc_i, uc_i) (larger magnitude if both).
 * y must be sign-consistent with the row bounds (y_i <= 0 where lc_i = -inf,
 * y_i >= 0 where uc_i = +inf), as the solver's points are: the term of an
 * infinite bound is dropped, so the wrong sign there goes unreported.
 * out[0] ||r_p||, out[1] ||r_d||, out[2] p, out[3] d, out[4] |p-d|,
 * out[5] rel.  Needs mpax_prepare. */
mpax_status mpax_kkt(mpax_problem* prob, const double* x, const double* y, mpax_mem_kind kind,
                     double* out);

/* ---- Differentiation of the returned solution ------------------------------ */

/* Reduced costs lam = Q x + c - A^T y (unscaled, n entries) at the point
 * mpax_get_solution returns: the multipliers of the variable bounds (eq. 1's
 * dual, Sec. 2). */
mpax_status mpax_get_reduced_cost(mpax_problem* prob, double* lam, mpax_mem_kind kind);

/* Gradients of an LP's optimal value at the returned point (x, y) of the last
 * mpax_solve, by the envelope theorem (the paper differentiates LPs through
 * surrogate losses, Sec. 3.4; the value gradient is what those losses use):
 * dc = x, dlc = y^+, duc = -y^-, dl = lam^+, du = -lam^- with lam = c - A^T y,
 * all unscaled.  Any output may be NULL; lengths n (dc, dl, du), m (dlc, duc). */
mpax_status mpax_lp_value_grad(mpax_problem* prob, double* dc, double* dlc, double* duc,
                               double* dl, double* du, mpax_mem_kind kind);

/* Implicit adjoint of a strictly convex QP's returned solution x* (Q = diag(D)
 * + F F^T) for a loss with gradient g = dL/dx* (n).  On the active set at x*
 * (free variables: strictly inside the box, or at a bound with multiplier
 * |lam_j| <= 1e-7 (1 + ||c||_inf), bound distance tested at 1e-7 (1 + |bound|);
 * active rows: equalities and rows with y_i != 0) it solves
 *     [[Q_FF, A_RF^T], [A_RF, 0]] [w; v] = [g_F; 0]
 * by MINRES (relative residual tol, at most max_iter iterations) with the
 * library's SpMVs in FP64, and returns dc = -w (free entries, else 0),
 * db = v (active rows, else 0; n.b. b is the row bound of equality rows),
 * dD = -w x* (free entries; dD may be NULL).  info (HOST, 2 doubles,
 * nullable) receives the iteration count and the final relative residual. */
mpax_status mpax_qp_adjoint(mpax_problem* prob, const double* g, double* dc, double* db,
                            double* dD, double tol, int32_t max_iter, mpax_mem_kind kind,
                            double* info);

/* Gradients of a QP solve by differentiating through its iterations (Sec. 3.4:
 * the paper differentiates QPs by unrolling Algorithm 2).  The last mpax_solve
 * of `prob` must have run with record_tape = 1 and precision FP64.  For the
 * loss L = gx . x + gy . y at its returned point (x, y), the derivative is
 * taken along the path that solve took: its restarts, step sizes (primal
 * weight), scaling and stopping point held fixed, each projection with
 * derivative 1 strictly inside its interval and 0 at or beyond a bound (and 1
 * in the bound it returned).  Outputs, all nullable: dc, dl, du, dD (n),
 * dlc, duc (m); an equality row's dL/db is dlc + duc.  gy is nullable (zero).
 * Cost: every block of the path is replayed once and run backwards, about two
 * forward solves.  MPAX_ERR_NOT_SOLVED without a taped solve. */
mpax_status mpax_qp_unrolled_grad(mpax_problem* prob, const double* gx, const double* gy,
                                  double* dc, double* dlc, double* duc, double* dl,
                                  double* du, double* dD, mpax_mem_kind kind);

/* ---- Ragged batch of independent LPs ---------------------------------------- */

/* B independent LPs of problem (1) (Q = 0), of any sizes, solved together in
 * one persistent kernel launch (the paper's batched solving, Sec. 3.2, without
 * its same-shape restriction).  Instance b owns rows [m_off[b], m_off[b+1]) and
 * columns [n_off[b], n_off[b+1]) (m_off, n_off: B+1 int64 entries starting at
 * 0).  row_ptr is the CSR row pointer over all rows (sum m + 1 entries, global
 * nonzero offsets); col_idx are column indices LOCAL to each instance
 * (0 <= col < n_b); val and the vectors are packed in instance order.
 * Validation and ownership as mpax_lp_create.  Every instance gets its own
 * scaling, step sizes, primal weight, restarts and termination. */
typedef struct mpax_batch mpax_batch;

typedef struct mpax_batch_stats {
  int32_t B;
  int32_t n_optimal;              /* instances that met the relative KKT test */
  int64_t iterations_total, iterations_max, restarts_total;
  double rel_kkt_max;
  double instance_seconds_p50;    /* per-instance device time (CTA start to finish) */
  double instance_seconds_p99;
  double instance_seconds_max;
  double solve_seconds;           /* whole mpax_batch_solve, host wall clock */
  int64_t kernel_launches;
  int32_t fp64_instances;         /* ragged batch, MIXED with fp64_continuation: instances
                                     whose FP32 run stalled and were continued in FP64;
                                     shared batch: instances still running when the
                                     products switched from BF16x3 to FP32 */
} mpax_batch_stats;

mpax_status mpax_lp_batch_create(int32_t B, const int64_t* m_off, const int64_t* n_off,
                                 const int64_t* row_ptr, const int32_t* col_idx,
                                 const double* val, const double* c, const double* lc,
                                 const double* uc, const double* l, const double* u,
                                 mpax_mem_kind kind, void* cuda_stream, mpax_batch** out);
/* Options as mpax_solve (reflection_gamma must be 1).  The batch runs as one
 * persistent launch; time_limit is measured on the device clock from the start
 * of that launch and is capped at 600 s, so the launch always ends (instances
 * still running then finish with MPAX_TERM_TIME_LIMIT).  In MIXED precision with
 * fp64_continuation, instances whose FP32 KKT error stops improving (the rule of
 * mpax_options.fp64_continuation, per instance) are continued from their FP32
 * point in a second, FP64 launch over those instances only.  An instance's two
 * gathered vectors sit in its CTA's shared memory when m_b + n_b <= 51,200
 * (FP32) or 25,600 (FP64), and in global memory otherwise (same arithmetic,
 * slower gathers); the shared pool of a launch is sized to the largest instance
 * of that launch that fits. */
mpax_status mpax_batch_solve(mpax_batch* batch, const mpax_options* opts);
/* Returned points (x^, y^) of every instance, packed like the inputs. */
mpax_status mpax_batch_get_solution(const mpax_batch* batch, double* x, double* y,
                                    mpax_mem_kind kind);
/* Summary, and (each pointer nullable, HOST memory, B entries) per-instance
 * termination, iterations, relative KKT error, primal objective, device seconds. */
mpax_status mpax_batch_get_stats(const mpax_batch* batch, mpax_batch_stats* stats,
                                 int32_t* status, int64_t* iterations, double* rel_kkt,
                                 double* primal_obj, double* seconds);
void mpax_batch_destroy(mpax_batch* batch);

/* B copies of ONE LP's constraints -- min c_b^T x s.t. lc <= A x <= uc,
 * l <= x <= u, A m x n in CSR as mpax_lp_create takes it -- as a ragged batch
 * whose instances differ only in their costs (the batched solving of Sec. 3.2
 * over a shared sparse feasible set, as in the paper's shortest-path
 * experiment, Sec. 4).  The B copies are built on the device from one copy of
 * the set; the costs start at zero (set them with mpax_batch_set_costs).
 * Errors as mpax_lp_batch_create; B * nnz, B * m, B * n must be < 2^31. */
mpax_status mpax_lp_batch_create_replicated(int32_t B, int32_t m, int32_t n, int64_t nnz,
                                            const int64_t* row_ptr, const int32_t* col_idx,
                                            const double* val, const double* lc,
                                            const double* uc, const double* l, const double* u,
                                            mpax_mem_kind kind, void* cuda_stream,
                                            mpax_batch** out);
/* Replace every instance's cost vector (packed like the batch's inputs: sum n_b
 * entries; for a replicated batch row b of a B x n row-major matrix).  The next
 * solve uses them. */
mpax_status mpax_batch_set_costs(mpax_batch* batch, const double* c, mpax_mem_kind kind);
/* Primal objective c_b^T x_b of every instance's returned point (B entries). */
mpax_status mpax_batch_get_objective(const mpax_batch* batch, double* v, mpax_mem_kind kind);
/* The SPO+ surrogate loss (Sec. 3.4: the paper trains LP decision models through
 * surrogate losses; SPO+ is the one of Elmachtoub and Grigas, 2022) of predicted
 * costs c_hat against true costs c_true, all instances at once:
 *   loss_b = -min_x (2 c_hat_b - c_true_b)^T x + 2 c_hat_b^T x*_b - z*_b,
 *   grad_b = 2 (x*_b - x~_b),  x~_b the returned minimiser of the first term,
 * a subgradient of loss_b in c_hat_b.  x*_b, z*_b (the true costs' optimum and
 * value) are inputs.  The call writes 2 c_hat - c_true into the batch's costs,
 * solves with `opts` (as mpax_batch_solve) and forms loss and grad in FP64 on
 * the device.  c_hat, c_true, x_true, grad: packed like the costs; z_true, loss:
 * B entries; all in `kind` memory (DEVICE: nothing crosses to the host but the
 * solve's own control words).  Afterwards the batch holds the solve of
 * 2 c_hat - c_true (mpax_batch_get_solution gives x~). */
mpax_status mpax_batch_spo_plus(mpax_batch* batch, const mpax_options* opts,
                                const double* c_hat, const double* c_true,
                                const double* x_true, const double* z_true, double* loss,
                                double* grad, mpax_mem_kind kind);

/* ---- Batch of LPs sharing one dense constraint matrix ----------------------- */

/* B LPs  min c_k^T x  s.t.  lc <= A x <= uc, l <= x <= u  with one dense A
 * (m x n, FP32, row-major) and per-instance costs C (B x n, row-major: row k is
 * c_k); lc, uc (m) and l, u (n) are shared.  Stacking the iterates as columns
 * makes both products of an iteration dense GEMMs (the paper's batched solving,
 * Sec. 3.2, with a shared matrix); they run on the tensor cores as three BF16
 * GEMMs with FP32 accumulation (BF16x3 split of the scaled matrix and of the
 * iterates), or, with fp32_products = 1, as one FP32 GEMM on the FP32 pipes.
 * Every instance has its own step sizes, primal weight, restarts and
 * termination (Algorithm 1).  Arrays are copied at create. */
typedef struct mpax_shared mpax_shared;
mpax_status mpax_lp_shared_create(int32_t m, int32_t n, int32_t B, const float* A,
                                  const double* C, const double* lc, const double* uc,
                                  const double* l, const double* u, mpax_mem_kind kind,
                                  void* cuda_stream, mpax_shared** out);
/* Options as mpax_solve (reflection_gamma must be 1); time_limit is checked on
 * the host clock at each KKT check.  With BF16x3 products and fp64_continuation,
 * once an unfinished instance's KKT error stops improving (the rule of
 * mpax_options.fp64_continuation, per instance) the rest of the solve forms its
 * products in FP32; mpax_shared_get_stats then reports the instances still
 * running at that point in fp64_instances. */
mpax_status mpax_shared_solve(mpax_shared* sh, const mpax_options* opts, int32_t fp32_products);
/* X: B x n (row k = x of instance k), Y: B x m, unscaled; either may be NULL. */
mpax_status mpax_shared_get_solution(const mpax_shared* sh, double* X, double* Y,
                                     mpax_mem_kind kind);
/* As mpax_batch_get_stats (seconds = host time from solve start to the check at
 * which the instance finished); gemm_info (HOST, 9 doubles, nullable) receives
 * the count of product launches, their flops, ||A~||_2, the K block (64 or 32)
 * of the dual and the primal product's pipeline (each direction's shape is
 * chosen by timing both on the first solve of each (m, n, B) in the process),
 * and, when the solve ran with profile_kernels = 1, the average milliseconds of
 * one iteration product launch, dual (A~ X) then primal (A~^T Y), from CUDA
 * events on the solve's stream (0 otherwise); then the host seconds of the
 * solve's preparation (scaling, BF16 splits, plans, norm estimate) and the
 * rounds of its power iteration (9 doubles in all). */
mpax_status mpax_shared_get_stats(const mpax_shared* sh, mpax_batch_stats* stats,
                                  int32_t* status, int64_t* iterations, double* rel_kkt,
                                  double* primal_obj, double* seconds, double* gemm_info);
void mpax_shared_destroy(mpax_shared* sh);
/* Replace the B cost vectors (B x n, row-major) of a shared-matrix batch; the
 * matrix, its scaling inputs and the bounds stay. */
mpax_status mpax_shared_set_costs(mpax_shared* sh, const double* C, mpax_mem_kind kind);
/* Primal objective c_k^T x_k of every instance's returned point (B entries). */
mpax_status mpax_shared_get_objective(const mpax_shared* sh, double* v, mpax_mem_kind kind);
/* SPO+ over the shared feasible set, as mpax_batch_spo_plus (C_hat, C_true,
 * X_true, grad: B x n row-major; z_true, loss: B), solving with
 * mpax_shared_solve(opts, fp32_products). */
mpax_status mpax_shared_spo_plus(mpax_shared* sh, const mpax_options* opts,
                                 int32_t fp32_products, const double* C_hat,
                                 const double* C_true, const double* X_true,
                                 const double* z_true, double* loss, double* grad,
                                 mpax_mem_kind kind);

/* One product of the shared-matrix batch on its own (Sec. 3.2: with the
 * iterates of B instances as the columns of a matrix, the two products of an
 * iteration are dense matrix products):
 *   D (M x N) = A_op (M x K) . V^T,   V: N x K (row n = the vector of instance n),
 * A_op = A stored row-major [M][K] (a_mn_major = 0; the dual step's A~ X) or
 * A^T of an A stored [K][M] (a_mn_major = 1; the primal step's A~^T Y).  Both
 * FP32 operands are split x = x_hi + x_lo (x_hi = bf16(x), x_lo = bf16(x - x_hi))
 * and D = A_hi V_lo + A_lo V_hi + A_hi V_hi is formed on the tensor cores
 * (tcgen05, FP32 accumulation), the kernel the shared batch uses.  Its error
 * against the exact product is at most (3 * 2^-18 + (3K + 2) * 2^-24) *
 * sum_k |A_op,mk| |V_nk| per entry.  D is [N][M] (row n = instance n).
 * tile_k: K block of the kernel's pipeline, 64 (two stages) or 32 (four
 * stages); 0 = 32.  Both give the same sums in the same order.  All pointers in
 * `kind` memory; the call allocates its BF16 operand copies and returns when D
 * is written.  Errors: MPAX_ERR_INVALID_ARGUMENT, MPAX_ERR_OUT_OF_MEMORY,
 * MPAX_ERR_CUDA, MPAX_ERR_DEVICE_TIMEOUT (a bounded wait of the kernel gave
 * up). */
mpax_status mpax_dense_bf16x3(int32_t M, int32_t N, int32_t K, int32_t a_mn_major,
                              int32_t tile_k, const float* A, const float* V, float* D,
                              mpax_mem_kind kind, void* cuda_stream);

/* ---- Evaluation without device allocation --------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc: code that runs inside a device-memory pool or budget
 * it does not own (a framework allocator, a serving process with a fixed
 * reservation), or that must not allocate while a stream is being captured.
 *
 * It returns what mpax_kkt returns (same definitions, out[0..5]) for the LP
 * min c^T x s.t. lc <= A x <= uc, l <= x <= u at the point (x, y), computed
 * directly on caller-owned DEVICE arrays, without a problem handle and without
 * allocating anything: no cudaMalloc, no cudaFree, no allocating library call.
 * The caller passes A and its transpose as CSR (int64 row pointers, int32
 * columns sorted within each row, FP64 values; row_ptr has m+1 entries,
 * row_ptr_t has n+1), the vectors (c, l, u, x: n; lc, uc, y: m) and `out`
 * (6 doubles of device memory).  The work is queued on `cuda_stream` (NULL =
 * legacy default stream) and the call returns without waiting for it.
 *
 * y must be sign-consistent with the row bounds (y_i <= 0 where lc_i = -inf,
 * y_i >= 0 where uc_i = +inf), as every point the solver returns is: the dual
 * objective drops the term of an infinite bound, so a y of the wrong sign there
 * would go unreported (mpax_kkt takes the same convention).
 *
 * Scratch: the per-block partial sums live in one static device array of
 * 3.5 MiB, held by every GPU that loads the library until the process exits.
 * Its size is the limit: m and n must each be at most 16,777,216; larger sizes
 * return MPAX_ERR_UNSUPPORTED with a message.  Every slot read by a call is
 * written earlier in the same call, so nothing needs clearing between calls,
 * but all calls share the array: calls whose device work overlaps (on
 * different streams, or from different host threads) race and give wrong
 * results.  The first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream capture.
 * Errors: MPAX_ERR_INVALID_ARGUMENT (negative size, NULL pointer),
 * MPAX_ERR_UNSUPPORTED (size limit, device index >= 64), MPAX_ERR_CUDA. */
mpax_status mpax_lp_kkt_noalloc(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                                const int32_t* col_idx, const double* val,
                                const int64_t* row_ptr_t, const int32_t* col_idx_t,
                                const double* val_t, const double* c, const double* lc,
                                const double* uc, const double* l, const double* u,
                                const double* x, const double* y, double* out,
                                void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPAX_H_ */
