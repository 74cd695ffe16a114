/*
 * scylla.h -- C ABI of a GB300 (sm_103a) implementation of the hot path of the
 * Scylla primal heuristic (Mexi, Shamsi, Besancon, Le Bodic, arXiv 2307.03466):
 * the matrix-free PDHG solve of the LP relaxation that each feasibility-pump
 * round re-runs after its objective update (Algorithm 1), with fix-and-propagate
 * (Section 2.3) on the host.
 *
 * Problem (Algorithm 1, input; generalised to two-sided rows):
 *     min c^T x   s.t.   row_lo <= A x <= row_hi,   col_lo <= x <= col_hi,
 *     x_j integer for is_integer[j] = 1.
 * The paper's  A x >= b  is the case row_lo = b, row_hi = +INFINITY.
 *
 * Conventions for every call:
 *   - Return value: SCYLLA_OK (0) or a negative SCYLLA_ERR_* code.  Solver
 *     outcomes (converged, iteration limit, found, ...) are reported in result
 *     structs, never as error codes.  Nothing aborts or throws across the ABI.
 *   - A call whose comment lists no errors (the accessors and resets) returns
 *     SCYLLA_ERR_INVALID_ARG for a null handle, a null required pointer or an
 *     index out of range, and SCYLLA_ERR_CUDA when a CUDA call fails.
 *   - scylla_last_error() gives a message for the last failing call on the
 *     calling thread.
 *   - Host pointers are caller-owned, read during the call only, and copied.
 *     Arrays are dense, contiguous, of the stated length.  Pointers documented
 *     as "device" must point to memory of the device that was current when the
 *     handle was created.
 *   - A handle may be used by one host thread at a time.
 *   - Infinite bounds are IEEE +-INFINITY.  NaN is rejected everywhere.
 */
#ifndef SCYLLA_H
#define SCYLLA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (return values) ------------------------------------------ */
#define SCYLLA_OK 0
#define SCYLLA_ERR_INVALID_ARG (-1) /* malformed input; nothing was changed */
#define SCYLLA_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define SCYLLA_ERR_OOM (-3)         /* device or host allocation failed */
#define SCYLLA_ERR_TIMEOUT (-4)     /* a time limit expired inside the call */
#define SCYLLA_ERR_UNSUPPORTED (-6) /* valid input beyond a documented limit */

/* ---- PDHG solve status (scylla_pdhg_result.status) ------------------------ */
#define SCYLLA_CONVERGED 0  /* relative KKT error <= tol (Section 2.2) */
#define SCYLLA_ITER_LIMIT 1 /* k reached the iteration limit (Algorithm 1) */
#define SCYLLA_STALLED 2    /* rounding of x unchanged over stall_checks checks */
#define SCYLLA_NUMERICAL 3  /* NaN/Inf met in a step-size or KKT reduction */
#define SCYLLA_DEVICE_TIMEOUT 4 /* a bounded device-side wait ran out (the call returns SCYLLA_ERR_TIMEOUT) */
#define SCYLLA_INFEASIBLE 5 /* a dual ray proved the LP infeasible (scylla_params.infeasibility_checks) */

/* ---- run status (scylla_run_result.status) -------------------------------- */
#define SCYLLA_FOUND 0
#define SCYLLA_NOT_FOUND 1

/* ---- precision of the bulk PDHG iteration --------------------------------- */
#define SCYLLA_PREC_FP64 0  /* values, vectors and accumulation in FP64 */
#define SCYLLA_PREC_MIXED 1 /* FP32 SpMVs/vector updates; FP64 KKT, restarts, refinement */

/* CSR matrix with m rows and n columns.  rowptr has m+1 entries, rowptr[0] = 0,
 * non-decreasing, rowptr[m] = nnz; cols[p] in [0, n), strictly increasing within
 * each row (no duplicates); vals finite. */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* rowptr;
  const int32_t* cols;
  const double* vals;
} scylla_csr;

/* Parameters.  scylla_default_params() fills the paper's values where the paper
 * gives them (alpha, eps1, beta, eps_floor: Algorithm 1 and Section 2.2) and
 * PDLP's customary values for the rules the paper delegates to PDLP
 * (Section 2.1: step size, restarts, preconditioning). */
typedef struct {
  int32_t precision;            /* SCYLLA_PREC_FP64 (default) or SCYLLA_PREC_MIXED */
  int32_t n_check;              /* attempts between KKT checks (64) */
  int32_t ruiz_iters;           /* Ruiz equilibration passes (10) */
  int32_t pock_chambolle;       /* Pock-Chambolle alpha=1 scaling after Ruiz (1) */
  int32_t adaptive_step;        /* 1: adaptive step size; 0: fixed eta = f/||A~||_F (1) */
  int32_t restarts;             /* KKT-based restarts to current/average iterate (1) */
  int32_t primal_weight_update; /* update omega at restarts (1) */
  int32_t stall_checks;         /* stop when round(x_I) is unchanged for this many checks; 0 = off (0) */
  int32_t aux_general_integers; /* add l1-distance auxiliary columns/rows for general integers (1) */
  int32_t use_graph;            /* 3: one persistent cooperative kernel runs the whole solve (grid
                                   barriers between phases; falls back to 1 where it cannot be
                                   co-resident); 1: one CUDA graph per n_check attempts, replayed by a
                                   pipelined host loop; 2: a single graph with a device-side while
                                   loop; 0: direct launches (1) */
  double fixed_step_factor;     /* f of the fixed-step mode (0.9) */
  double beta_sufficient;       /* restart if KKT <= 0.2 KKT_last_restart */
  double beta_necessary;        /* ... or <= 0.8 KKT_last_restart and KKT grew since the last check */
  double beta_artificial;       /* ... or attempts since restart >= 0.36 attempts */
  double pw_smoothing;          /* theta of the primal weight update (0.5) */
  double step_reduction_exp;    /* 0.3 */
  double step_growth_exp;       /* 0.6 */
  /* outer loop (scylla_run) */
  double alpha;                 /* 0.9 (Algorithm 1) */
  double eps1;                  /* 0.01 (Section 2.2) */
  double beta;                  /* 0.98 (Section 2.2) */
  double eps_floor;             /* 1e-8 (Section 2.2) */
  int64_t max_rounds;           /* pump rounds K (100) */
  int64_t iter_limit;           /* PDHG attempts per solve inside scylla_run (20000) */
  int64_t total_iter_cap;       /* PDHG attempts over the whole run (1e9) */
  int32_t run_stall_checks;     /* stall_checks used by scylla_run's solves (5) */
  int32_t trace_capacity;       /* attempts recorded by the decision trace of each solve; 0 = off (0) */
  uint64_t seed;                /* perturbation random stream (0) */
  double time_limit_s;          /* wall-clock limit of scylla_run, <= 0 for none (0) */
  double device_wait_limit_s;   /* bound of every device-side barrier wait (5) */
  int32_t pdl;                  /* launch the per-attempt kernels with programmatic dependent launch, so
                                   each one is resident before its predecessor ends (1) */
  int32_t prefetch;             /* form of the per-attempt kernels. 0: automatic (4 when A, A^T and the
                                   vectors fit in half of the L2 cache, else 2); 1: 32-row tiles, each
                                   warp loading its first tile before the wait on the preceding kernel;
                                   2: wide tiles of up to 128 rows, plain loads; 3: wide tiles staged in
                                   shared memory by bulk copies; 4: 32-row tiles, plain loads; 5 (FP32-mixed
                                   only): 32-row tiles, the warp's next tile staged in shared memory by
                                   asynchronous copies (0) */
  int32_t host_transpose;       /* 1: build the stored transpose A^T on the host threads; 0: on the device,
                                   a stable radix sort of the nonzeros by column (0) */
  /* continuous repair inside scylla_run (see scylla_repair; not part of the paper's
     Algorithm 1, so off by default) */
  int64_t repair_iters;         /* attempt limit of each repair (all its rounds); 0 = no repair (0) */
  double repair_tol;            /* rel-KKT target of each repair solve (1e-7) */
  int32_t repair_rounds;        /* solves of one repair, with the violated rows shifted in between (8) */
  int32_t distance;             /* distance of the objective update: 1 = l1 (Algorithm 1; auxiliary columns
                                   for general integers), 2 = l2 (the conclusion's alternative: a diagonal
                                   quadratic objective, no auxiliary columns) (1) */
  int32_t batch_launch;         /* batched solve: 0 automatic (at create, n_check attempts in each of 1, 2 and,
                                   FP32-mixed, 3 are timed and the fastest is kept); 1 one CUDA graph
                                   per n_check attempts, each phase a launch over a static deal of the tiles;
                                   2 the attempts between checks in one persistent cooperative launch whose
                                   warps take tiles from a shared queue over the LPs still running, the
                                   queue compacted at every check; 3 (FP32-mixed) as 1, each warp's next
                                   tile staged in shared memory by asynchronous copies (0) */
  int32_t autotune;             /* with prefetch = 0: 1 times the 32-row, wide-tile and (FP32) asynchronous-copy forms of the
                                   per-attempt kernels on the handle's own matrix at create and keeps the
                                   faster for each of the two kernels (the choice is kept per matrix shape
                                   for the process); 0 takes the L2-size rule (1) */
  int32_t infeasibility_checks; /* 1: at every check of a single-LP solve, test a candidate dual ray (the
                                   change of y since an earlier check) and end the solve SCYLLA_INFEASIBLE
                                   when it proves the LP infeasible (scylla_get_certificate); the
                                   persistent form (use_graph = 3) then runs as 1.  Batched solves reject
                                   it; fan-outs do not test.  (0) */
  int32_t dual_form;            /* with prefetch = 1..4: the dual per-attempt kernel's form, numbered as
                                   prefetch, when it differs from the primal's; 0 the same (0) */
} scylla_params;

typedef struct {
  int32_t status;        /* SCYLLA_CONVERGED / ITER_LIMIT / STALLED / NUMERICAL / INFEASIBLE */
  int32_t used_average;  /* 1 if the returned point is the averaged iterate */
  int64_t iterations;    /* step attempts k of this solve */
  int64_t accepted, rejected, restarts;
  double eps_p, eps_d, eps_g, rel_kkt; /* relative residuals of the returned point */
  double pobj, dobj;     /* primal/dual objective (with the objective offset) */
  double eta, omega;     /* step size and primal weight after the solve */
  double seconds;        /* device time of the solve (CUDA events) */
  int64_t launches;      /* kernel launches issued, including ones that returned early */
  int32_t kernel_form;   /* form of the primal per-attempt kernel (scylla_params.prefetch's numbering: 4
                            32-row tiles, 1 32-row with prefetch, 2 wide tiles, 3 staged wide tiles); 0 for
                            the batched and fan-out solves */
  int32_t kernel_form_dual; /* form of the dual per-attempt kernel, numbered alike */
} scylla_pdhg_result;

typedef struct {
  int32_t status;           /* SCYLLA_FOUND / SCYLLA_NOT_FOUND */
  int32_t found_by;         /* 1: rounded LP point (Algorithm 1 first test), 2: fix-and-propagate,
                               3: continuous repair of the fix-and-propagate point */
  int64_t rounds;           /* pump rounds K performed */
  int64_t total_iterations; /* PDHG attempts over all rounds */
  int64_t perturbations;    /* rounds in which cycling was detected */
  double objective;         /* c^T x of the returned point */
  double seconds, seconds_pdhg, seconds_fixprop;
} scylla_run_result;

typedef struct {
  int32_t status;       /* SCYLLA_FOUND when the repaired point passes scylla_check_feasible */
  int32_t pdhg_status;  /* status of the last repair solve (SCYLLA_CONVERGED / ITER_LIMIT / ...) */
  int64_t iterations;   /* PDHG attempts of all rounds */
  int32_t rounds;       /* solves performed */
  int32_t shifted_rows; /* rows whose working bounds were moved, over all rounds */
  double rel_kkt;       /* relative KKT error of the last solve's point (on its working bounds) */
  double objective;     /* c^T x of the returned point */
  double seconds;       /* device time of the solves */
} scylla_repair_result;

typedef struct scylla_lp scylla_lp; /* opaque; owns all device and host copies */

/* Fill *p with the defaults listed above. */
void scylla_default_params(scylla_params* p);

/* Validate and copy the MIP, add the auxiliary distance columns (Section 4: the l1
 * distance on general integers needs auxiliary variables), build the transposed
 * CSR so that A^T y is a row gather (Algorithm 1, primal step), precondition on
 * the GPU (Section 2.1: PDLP's diagonal preconditioning), and set the initial
 * point x = proj_[l,u](0), y = 0 (Algorithm 1, initialisation).
 *   c, col_lo, col_hi, is_integer: host, length A->n.  row_lo, row_hi: host,
 *   length A->m.  p: NULL for defaults.  cuda_stream: a cudaStream_t whose prior
 *   work is ordered before each call of this handle, or NULL.
 * Errors: INVALID_ARG (see scylla_csr; also lo > hi, NaN, integer column with a
 * fractional finite bound, is_integer not 0/1), UNSUPPORTED (nnz or a dimension
 * >= 2^31 - 64), OOM, CUDA.  On error *out is NULL. */
int scylla_lp_create(const scylla_csr* A, const double* c, const double* row_lo, const double* row_hi,
                     const double* col_lo, const double* col_hi, const uint8_t* is_integer,
                     const scylla_params* p, void* cuda_stream, scylla_lp** out);

/* Free every resource of the handle.  NULL is a no-op. */
void scylla_lp_destroy(scylla_lp* lp);

/* Dimensions of the LP the solver iterates on (original plus auxiliary). */
int scylla_lp_dims(const scylla_lp* lp, int64_t* m_total, int64_t* n_total, int64_t* nnz_total,
                   int64_t* n_aux);

/* PDHG on the GPU (Algorithm 1 inner loop; Sections 2.1-2.2) from the handle's
 * current primal-dual pair (a warm start, Section 2.1), until the relative KKT
 * error of the current or averaged iterate is <= tol, or k = iter_limit, or the
 * stall rule fires.  The returned point becomes the handle's current pair.
 * tol >= 0; iter_limit >= 0.  Errors: INVALID_ARG, CUDA. */
int scylla_pdhg_solve(scylla_lp* lp, double tol, int64_t iter_limit, scylla_pdhg_result* out);

/* Objective update of Algorithm 1 / Section 2.4 for round K >= 1 around the
 * integer point xhat (host, length n original; entries on integer columns must be
 * integral and inside their bounds).  Keeps x, y, eta, omega (warm start).
 * Errors: INVALID_ARG, CUDA. */
int scylla_set_objective(scylla_lp* lp, const double* xhat, int32_t K);
/* (With p.distance = 2 the update is the l2 one instead: c_hat_j = alpha^K s c_j -
 * (1 - alpha^K) xhat_j and q_j = 1 - alpha^K on the integer columns, c_hat_j =
 * alpha^K s c_j and q_j = 0 elsewhere, offset (1 - alpha^K)/2 sum xhat_j^2 over the
 * integer columns: alpha^K s c^T x + (1 - alpha^K)/2 ||x_I - xhat_I||^2 as a
 * diagonal quadratic objective, see scylla_set_qp_objective.) */

/* Diagonal quadratic objective on the original columns (the conclusion's remark that
 * PDHG, as in PDLP, takes objectives with a diagonal Hessian):
 *     min c^T x + 1/2 x^T diag(q) x + offset   over the same constraints.
 * c, q: host, length n (q_j >= 0, finite).  The primal step becomes the closed-form
 * prox x' = proj_[l,u]((x + tau (A^T y - c)) / (1 + tau q)) in the scaled space, and
 * the KKT error uses the reduced cost c + q x - A^T y and the objectives
 * +-1/2 x^T Q x; an all-zero q is the LP exactly.  Keeps the iterate (warm start).
 * Auxiliary columns keep their cost and get q = 0.  The batched and fan-out solves
 * take LPs only.  Errors: INVALID_ARG (null, non-finite c or offset, q < 0 or
 * non-finite), CUDA. */
int scylla_set_qp_objective(scylla_lp* lp, const double* c, const double* q, double offset);

/* Current objective c_hat (host, length n_total) and offset, unscaled. */
int scylla_get_objective(const scylla_lp* lp, double* c_hat, double* offset);

/* The whole heuristic (Algorithm 1): PDHG -> MIP-feasibility test -> fix-and-
 * propagate -> feasibility test -> cycle handling -> objective update, with the
 * tolerance schedule of Section 2.2.  With p.repair_iters > 0 a fix-and-propagate
 * point that fails the test is given to scylla_repair (p.repair_tol, p.repair_iters)
 * before the cycle handling.  x_out (host, length n original) receives the solution
 * when out->status == SCYLLA_FOUND; every returned point passed
 * scylla_check_feasible.  Errors: INVALID_ARG, OOM (host), CUDA, TIMEOUT (time limit hit). */
int scylla_run(scylla_lp* lp, double* x_out, scylla_run_result* out);

/* Current primal point, unscaled: host length n (original columns). */
int scylla_get_primal(const scylla_lp* lp, double* x);
/* Current dual point, unscaled: host length m (original rows). */
int scylla_get_dual(const scylla_lp* lp, double* y);
/* Same, device pointer of length n (original columns), FP64. */
int scylla_get_primal_device(const scylla_lp* lp, double* x_device);

/* Full iterate of the solved LP (original plus auxiliary), unscaled, host:
 * x length n_total, y length m_total; eta, omega may be NULL. */
int scylla_get_state(const scylla_lp* lp, double* x, double* y, double* eta, double* omega);
/* Replace the iterate (checkpoint/resume; Section 2.1 notes the PDLP state is the
 * primal-dual pair).  Same layout as scylla_get_state; eta, omega > 0. */
int scylla_set_state(scylla_lp* lp, const double* x, const double* y, double eta, double omega);

/* Cold restart: x = proj_[l,u](0), y = 0 (Algorithm 1 initialisation) and the step
 * size and primal weight chosen at create.  The objective is left as it is. */
int scylla_reset_state(scylla_lp* lp);

/* Measurement: run `attempts` PDHG attempts from the current pair (no tolerance
 * test; every n_check attempts the check kernels run as in a solve) as separate
 * launches on the handle's stream, with CUDA events around each launch, and write
 * the mean device time in milliseconds of each kernel to ms[0..3]: primal step,
 * dual step, column check, row check (0 where a kernel did not run).  The pair
 * moves on by those attempts. */
int scylla_time_kernels(scylla_lp* lp, int32_t attempts, double* ms);

/* Forms of the primal and the dual per-attempt kernels in use (numbered as
 * scylla_params.prefetch: 4 32-row tiles, 1 32-row with prefetch, 2 wide tiles, 3
 * staged, 5 asynchronous copies), the form the L2-size rule gives both, and the
 * create-time autotuner's device times per launch in ms, tune_ms[0..5] = primal and
 * dual of the 32-row form, of the wide form, and of the asynchronous-copy form (0
 * when it did not time them: a forced form, autotune = 0, FP64 for the last pair, or
 * the choice kept from an earlier handle of the same shape).  The autotuner picks
 * each kernel's form on its own.  Any output may be NULL. */
int scylla_kernel_form(const scylla_lp* lp, int32_t* form, int32_t* form_dual, int32_t* rule_form,
                       double* tune_ms);

/* Diagonal scaling A~ = diag(R) A diag(C) found at create: host, R length m_total,
 * C length n_total. */
int scylla_get_scaling(const scylla_lp* lp, double* R, double* C);

/* The stored transpose of the scaled matrix A~ that the primal step gathers over
 * (Section 2.1): host arrays colptr (n_total + 1), rows (nnz_total, ascending within
 * each column) and vals (nnz_total, FP64); any of the three may be null. */
int scylla_get_transpose(const scylla_lp* lp, int64_t* colptr, int32_t* rows, double* vals);

/* Fix-and-propagate (Section 2.3) on the original MIP, on the host.
 *   xbar: host, length n.  xhat, dom_lo, dom_hi: host outputs, length n.
 *   fixed_cols: host output, length n (may be NULL), receives the columns fixed
 *   by rounding in fixing order; *n_fixed their count (may be NULL).
 *   ignored_rows: host output, length m (may be NULL), 1 for rows ignored after
 *   emptying a domain.
 * The first call keeps, in the handle, the end state of the propagation of the
 * bounds alone (it depends only on the MIP); later calls start from it, with the
 * same results, until scylla_set_col_bounds or scylla_set_row_bounds drops it.
 * Errors: INVALID_ARG (null lp, xbar or xhat; NaN in xbar), OOM (host), CUDA (first
 * download of the host copies). */
int scylla_fix_and_propagate(const scylla_lp* lp, const double* xbar, double* xhat, double* dom_lo,
                             double* dom_hi, int32_t* fixed_cols, int64_t* n_fixed, uint8_t* ignored_rows);

/* Fix-and-propagate of K points at once (Section 2.3), e.g. the K LP points of a
 * fan-out solve, on the host threads.  Point k gives exactly what
 * scylla_fix_and_propagate gives for it; every point starts from the handle's kept
 * first propagation (computed first, on the calling thread).
 *   K >= 0.  xbar: host, K blocks of length n (point k at xbar + k n).
 *   xhat: host output, K blocks of length n.  dom_lo, dom_hi: host outputs, K blocks
 *   of length n, or NULL.  n_fixed: host output, K entries, or NULL.
 * Errors: INVALID_ARG (null lp, K < 0, null xbar or xhat with K > 0, NaN in xbar),
 * OOM (host), CUDA (first download of the host copies). */
int scylla_fix_and_propagate_many(const scylla_lp* lp, int32_t K, const double* xbar, double* xhat,
                                  double* dom_lo, double* dom_hi, int64_t* n_fixed);

/* Exact MIP-feasibility test of x (host, length n) on the original MIP
 * (Algorithm 1, both "MIP-feasible" tests): *feasible = 1 or 0.
 * Errors: INVALID_ARG (null), OOM (host), CUDA (first download of the host copies). */
int scylla_check_feasible(const scylla_lp* lp, const double* x, int32_t* feasible);

/* Test of a certificate that the original LP relaxation has no feasible point, by
 * weak duality (the LP solves Section 2.1 hands to PDLP can end in such a report):
 *     D(y) = sum_i min_{lo_i <= s_i <= hi_i} y_i s_i
 *          - sum_j max_{l_j <= x_j <= u_j} (A^T y)_j x_j
 * over the original rows and columns.  Every feasible x has
 * (first sum) <= y^T A x <= (second sum), so D(y) > 0 proves that none exists.
 *   y: host, length m (one multiplier per original row).
 *   *gap receives D(y), or -INFINITY when a term needs an infinite bound (y_i > 0
 *   with row_lo_i = -inf, (A^T y)_j > 0 with col_hi_j = +inf, or the mirror cases).
 * FP64 with compensated sums in a fixed order, on the host.
 * Errors: INVALID_ARG (null, a NaN or infinite entry of y), OOM (host), CUDA (first
 * download of the host copies). */
int scylla_farkas_gap(const scylla_lp* lp, const double* y, double* gap);

/* The dual ray tested at the last check of the last solve of a handle created with
 * scylla_params.infeasibility_checks = 1 (the solve's status is SCYLLA_INFEASIBLE when
 * the test proved the LP infeasible).
 * Detection (a reading of the LP solver Section 2.1 hands the relaxations to): at the
 * check after k = q n_check attempts (q >= 2) the candidate is y_k - y_a, where y_a is
 * the dual at the last earlier check whose q is a power of two, with every entry set
 * to 0 whose sign would need an infinite row bound.  The device computes D of the
 * ray (as in scylla_farkas_gap, over the rows and columns the solve iterates, in the
 * scaled space, each (A^T y)_j a compensated sum) and S, the sum of the absolute
 * values of D's terms; the solve ends SCYLLA_INFEASIBLE when D > 1e-9 S and (without
 * auxiliary distance rows) the host's test of the ray on the original data,
 * scylla_farkas_gap, gives D > 0; a ray that fails it ends the solve
 * SCYLLA_NUMERICAL.  On a feasible LP D <= 0 (weak duality), and 1e-9 S is far
 * above the rounding of D.
 *   y: host, length m of the original rows (may be null): the ray, unscaled, zero when
 *      no candidate was tested.  With auxiliary distance rows
 *      (aux_general_integers) the ray may weigh them too; y holds the original rows'
 *      entries only.  scylla_farkas_gap(lp, y) tests it on the original data.
 *   gap, scale (may be null): D and S as the device computed them; -INFINITY and 0
 *      when no candidate was tested, gap = -INFINITY when a term needed an infinite
 *      bound.
 * Errors: INVALID_ARG (null handle, or a handle created without
 * infeasibility_checks), CUDA. */
int scylla_get_certificate(const scylla_lp* lp, double* y, double* gap, double* scale);

/* Replace the bounds of the original columns (host, length n each), keeping the
 * matrix, its preconditioning, the objective and the iterate; the auxiliary columns
 * keep theirs.  The next solve projects onto the new box (Algorithm 1, primal step);
 * call scylla_reset_state for a cold start.  The host copies used by the propagation
 * and the feasibility test see the new bounds too.
 * Errors: INVALID_ARG (null, NaN, lo > hi, lo = +inf, hi = -inf, an integer column
 * with a fractional finite bound), CUDA. */
int scylla_set_col_bounds(scylla_lp* lp, const double* col_lo, const double* col_hi);

/* Bound propagation on the GPU: the activity-based tightening of fix-and-propagate
 * (Section 2.3) over the original rows, in rounds.  In a round every active row
 * (all rows in the first) derives, from the domains at the start of the round and
 * with the arithmetic of one visit of the sequential propagation, the bounds it
 * tightens; every column then takes the tightest of them.  A row whose activity
 * bounds exclude [lo, hi] or that would empty a domain is ignored from then on; a
 * column whose merged bounds cross by more than 1e-9 keeps its domain (a conflict).
 * The rows of changed columns are the next round's; it stops when there are none or
 * after max_rounds.  On integer data without ignored rows or conflicts the result is
 * the sequential propagation's fixpoint bit for bit (scylla_fix_and_propagate's
 * first step); on other data it can differ where the continuous thresholds make the
 * order matter.
 *   dom_lo, dom_hi: host, length n, the starting domains in, the propagated ones out.
 *   ignored_rows: host, length m, or NULL.  rounds, conflicts: outputs, or NULL.
 * Errors: INVALID_ARG (null, NaN, lo > hi, max_rounds < 1), OOM, CUDA. */
int scylla_propagate(scylla_lp* lp, double* dom_lo, double* dom_hi, uint8_t* ignored_rows, int64_t max_rounds,
                     int64_t* rounds, int64_t* conflicts);

/* Replace the bounds of the original rows (host, length m each), keeping the
 * matrix, its preconditioning, the objective and the iterate; auxiliary rows keep
 * theirs, and ||b|| of the relative KKT error follows the new bounds.
 * Errors: INVALID_ARG (null, NaN, lo > hi, lo = +inf, hi = -inf), CUDA. */
int scylla_set_row_bounds(scylla_lp* lp, const double* row_lo, const double* row_hi);

/* Continuous repair of an integer assignment.  The paper keeps the continuous part
 * of fix-and-propagate's point at the LP values (Section 2.3), which on mixed
 * problems often leaves rows violated; this re-solves the LP with the integer
 * columns fixed,
 *     min c^T x  s.t.  lo <= A x <= hi,  x_j = xhat_j (j integer),
 *                      l_j <= x_j <= u_j (j continuous),
 * by the same PDHG path (preconditioning, adaptive steps, restarts, FP64 checks;
 * Sections 2.1-2.2) on a second device copy of the original MIP that the handle
 * builds on first use (original objective, no auxiliary columns, the handle's PDHG
 * parameters, always FP64) and keeps until it is destroyed.  First the fixing is
 * propagated on the GPU (scylla_propagate, at most 1000 rounds): a row it ignores or
 * a conflict proves the fixed LP infeasible, and then no solve runs (rounds = 0,
 * x_out = xhat clamped to the bounds).  Otherwise up to
 * p.repair_rounds solves to rel-KKT <= tol, the first from the cold start, the next
 * ones warm: after each, the integer entries are set to xhat's exactly and the point
 * is given scylla_check_feasible's test; if it fails, every row whose activity
 * (FP64, in CSR order) exceeds an original bound has its working bound moved
 * inward by the excess plus the test's tolerance 1e-6 max(1, |bound|) (a row whose
 * working bounds would cross gets their midpoint), because a PDHG point at a
 * relative KKT error far below 1e-6 can still miss single rows by more than that.
 * iter_limit bounds the attempts of all rounds together.
 *   xhat: host, length n (integer entries integral within [l, u]; the others are
 *   ignored).  x_out: host, length n, receives the last point whatever the outcome.
 *   out: the test's verdict and the solves' figures (attempts and seconds summed).
 * Errors: INVALID_ARG (null, tol < 0, iter_limit < 0, xhat not integral within the
 * bounds of an integer column), OOM and CUDA from building the copy. */
int scylla_repair(scylla_lp* lp, const double* xhat, double tol, int64_t iter_limit, double* x_out,
                  scylla_repair_result* out);

/* Cycle handling of Section 2.3 on its own.  kind: 1 short cycle, 2 long cycle.
 * xhat: host in/out, length n; xbar: host, length n; K: round; seed: stream seed.
 * *flipped (may be NULL) receives the number of changed entries.
 * Errors: INVALID_ARG (null, kind not 1 or 2), OOM (host), CUDA (first download of
 * the host copies). */
int scylla_perturb(const scylla_lp* lp, double* xhat, const double* xbar, int32_t kind, int64_t K,
                   uint64_t seed, int64_t* flipped);

/* Decision trace of the last solve (enabled by params.trace_capacity > 0).
 *   steps: host, 4 * trace_capacity doubles; for attempt k = 1, 2, ... the record
 *   (eta used, eta_max of the adaptive rule, accepted 0/1, eta for the next
 *   attempt).  checks: host, 5 * trace_capacity doubles; for every check that
 *   neither terminated nor was the start-point evaluation, the record (k, restart
 *   0/1, candidate is the average 0/1, primal weight after the check, weighted KKT
 *   of the candidate).  *n_steps, *n_checks receive the record counts (capped at
 *   trace_capacity). */
int scylla_get_trace(const scylla_lp* lp, double* steps, int64_t* n_steps, double* checks, int64_t* n_checks);

/* Primal residual without any device allocation, for callers that cannot call
 * cudaMalloc: plugins whose host application hands them a fixed memory pool,
 * real-time loops that forbid allocator calls (cudaMalloc and cudaFree can block and
 * synchronise the device), processes sharing a GPU under a memory budget set
 * elsewhere.  The paper has no counterpart: this is a service entry point over the
 * same residual the solver's KKT check computes.
 *
 * Computes, on the caller's stream, for the caller's LP rows and point x:
 *   out[0] = ||A x - proj_[row_lo,row_hi](A x)||_2
 *   out[1] = out[0] / (1 + ||b||_2), b_i = the largest finite |row_lo_i|, |row_hi_i|
 * (eps_p of scylla_pdhg_result for the same point).
 *   m: rows, 1 <= m <= 2,097,152 (beyond that INVALID_ARG: the fixed scratch holds
 *   8192 block sums of 256 rows).  rowptr (int64, m+1), cols (int32), vals (double),
 *   x (double, the columns the CSR refers to), row_lo, row_hi (double, m), out
 *   (double, 2): all DEVICE pointers owned by the caller.  cuda_stream: a
 *   cudaStream_t or NULL.  The call is asynchronous: out is ready when the stream
 *   reaches it.
 * Scratch: one file-scope __device__ array of 128 KiB per device, held by every GPU
 * that loads the library until the process exits.  The first call on a device looks
 * the array's device address up (cudaGetSymbolAddress, with that device current)
 * and keeps it for the life of the process, so make that first call before any
 * stream capture, and do not use the entry point across a cudaDeviceReset (the kept
 * address would be stale).  Every call clears the array's arrival counter on its
 * stream (cudaMemsetAsync) before its kernel, so a call that failed part way leaves
 * nothing behind for the next one.  Every call shares the array, so calls that
 * overlap on the GPU race and must be serialised by the caller.  Nothing is
 * allocated, by this library or by any library it calls.
 * Errors: INVALID_ARG (sizes, null pointers), UNSUPPORTED (device ordinal >= 64),
 * CUDA. */
int scylla_primal_residual_noalloc(int64_t m, const int64_t* rowptr, const int32_t* cols, const double* vals,
                                   const double* x, const double* row_lo, const double* row_hi, double* out,
                                   void* cuda_stream);

/* ---- batched solve ---------------------------------------------------------
 * Many LP relaxations of uneven size solved together: one launch sequence walks a
 * shared list of warp tiles covering every LP (no tile spans two LPs), every LP has
 * its own step size, primal weight, restarts and termination (Sections 2.1-2.2
 * applied per LP), and a finished LP drops out while the others continue.  The LPs
 * have no integrality here (the batched form is the LP solve of the pump). */
typedef struct scylla_batch scylla_batch;

/* count >= 1 LPs; A[b] (host CSR), c[b], col_lo[b], col_hi[b] (host, length A[b].n),
 * row_lo[b], row_hi[b] (host, length A[b].m), each validated as in scylla_lp_create.
 * p: NULL for defaults (precision, n_check, step-size and restart parameters apply
 * to every LP).  Errors: INVALID_ARG (naming the LP), UNSUPPORTED (total size beyond
 * the 32-bit index range), OOM, CUDA. */
int scylla_batch_create(int32_t count, const scylla_csr* A, const double* const* c, const double* const* row_lo,
                        const double* const* row_hi, const double* const* col_lo, const double* const* col_hi,
                        const scylla_params* p, void* cuda_stream, scylla_batch** out);
void scylla_batch_destroy(scylla_batch* h);
/* PDHG on every LP from its current pair until each one's relative KKT error is
 * <= tol or it reaches iter_limit attempts.  results: host, count entries;
 * seconds (may be NULL): device time of the whole batch. */
int scylla_batch_solve(scylla_batch* h, double tol, int64_t iter_limit, scylla_pdhg_result* results,
                       double* seconds);
/* primal point of LP b, unscaled: host, length A[b].n */
int scylla_batch_get_primal(const scylla_batch* h, int32_t b, double* x);
/* dual point of LP b, unscaled: host, length A[b].m.  With scylla_batch_get_primal it
 * is the pair whose errors the LP's last result reports.  Errors: INVALID_ARG, CUDA. */
int scylla_batch_get_dual(const scylla_batch* h, int32_t b, double* y);
/* The launch form in use (*form, numbered as scylla_params.batch_launch: 1 graphs,
 * 2 the persistent work-queue launch, 3 graphs over asynchronous-copy tiles) and,
 * with batch_launch = 0, the ms of the n_check attempts each form took at create
 * (tune_ms[0] graphs, tune_ms[1] persistent, tune_ms[2] asynchronous-copy graphs;
 * 0 when not timed).  Either pointer may be NULL. */
int scylla_batch_info(const scylla_batch* h, int32_t* form, double* tune_ms);
/* Measurement: `attempts` attempts of every LP from its current pair (no tolerance
 * test) with the graph form's kernels as separate launches and CUDA events around
 * each; ms[0..2] receive the mean device time in milliseconds of the primal step,
 * the dual step and the step control.  Errors: INVALID_ARG, CUDA. */
int scylla_batch_time_kernels(scylla_batch* h, int32_t attempts, double* ms);
/* cold restart of every LP (x = proj_[l,u](0), y = 0, initial step sizes) */
int scylla_batch_reset_state(scylla_batch* h);

/* ---- K-objective fan-out ---------------------------------------------------
 * K pump objectives of one LP (Section 2.4: the objective update of round
 * round_K around K different rounding targets) solved together as sparse-times-
 * tall-skinny products, so A is read once per K objectives.  Every objective has
 * its own step size, primal weight, restarts and termination and starts from the
 * handle's current primal-dual pair (a warm start, Section 2.1).  The handle's
 * precision applies; in SCYLLA_PREC_MIXED the per-attempt step decisions run in
 * FP32 (as a single-LP solve's do) and the checks' sums over a row are compensated
 * FP32 pairs (about 2^-44 of the terms' magnitudes; residuals, objectives and norms
 * in FP64). */
typedef struct scylla_fanout scylla_fanout;

/* lp: a handle without auxiliary columns (created with aux_general_integers = 0);
 * it must outlive the fan-out, whose device data is its own except the shared
 * matrices.  K: 1..64.  targets: host, K blocks of length n (targets[k*n + j]);
 * integer entries integral within bounds.  Target k gives objective
 * alpha^round_K s c + (1 - alpha^round_K) g_k with g_kj = +1 (target at l_j), -1
 * (at u_j), 0 otherwise on integer columns.  Errors: INVALID_ARG, UNSUPPORTED
 * (auxiliary columns present), OOM, CUDA. */
int scylla_fanout_create(scylla_lp* lp, int32_t K, const double* targets, int32_t round_K, scylla_fanout** out);
void scylla_fanout_destroy(scylla_fanout* f);
/* PDHG for every objective until its relative KKT error is <= tol or it reaches
 * iter_limit attempts.  results: host, K entries; seconds (may be NULL): device
 * time of the whole fan-out. */
int scylla_fanout_solve(scylla_fanout* f, double tol, int64_t iter_limit, scylla_pdhg_result* results,
                        double* seconds);
/* primal point of objective k, unscaled: host, length n */
int scylla_fanout_get_primal(const scylla_fanout* f, int32_t k, double* x);
/* dual point of objective k, unscaled: host, length m (the rows of the LP; the
 * fan-out's LP has no auxiliary rows).  With scylla_fanout_get_primal it is the pair
 * whose errors the objective's last result reports.  Errors: INVALID_ARG, CUDA. */
int scylla_fanout_get_dual(const scylla_fanout* f, int32_t k, double* y);
/* every objective back to the handle's current pair, step size and primal weight */
int scylla_fanout_reset_state(scylla_fanout* f);
/* Tile-shape autotuner of the fan-out (run once by scylla_fanout_create).  Every
 * K-wide vector row has 64 slots; a tile shape sets how the SpMMs (primal over A^T,
 * dual over A) cover them: VEC consecutive objectives per lane and CHUNK slots per
 * sweep, so CHUNK / VEC lanes per row, 32 VEC / CHUNK rows per warp and 64 / CHUNK
 * sweeps over the matrix (two sweeps halve the part of the gathered vector in use
 * at a time).  Shapes: 1 = (4, 64), 2 = (2, 64), 3 = (4, 32), 4 = (2, 32); the
 * FP64 mode takes 2 and 4.  shape_primal, shape_dual: 0 times every valid shape on
 * this fan-out's own matrix and keeps the fastest, 1..4 forces one.  Every shape
 * gives identical results.  The objectives go back to the handle's pair (as
 * scylla_fanout_reset_state).  Errors: INVALID_ARG (an invalid shape), CUDA. */
int scylla_fanout_tune(scylla_fanout* f, int32_t shape_primal, int32_t shape_dual);
/* The tile shapes in use and the tuner's times: tune_ms (may be NULL) receives 8
 * values, ms per launch of the primal SpMM in shapes 1..4, then of the dual SpMM
 * (0 where a shape was not timed). */
int scylla_fanout_info(const scylla_fanout* f, int32_t* shape_primal, int32_t* shape_dual, double* tune_ms);
/* Measurement: `attempts` attempts of every objective from the current pairs (no
 * tolerance test; the checks run every n_check attempts as in a solve) as separate
 * launches with CUDA events around each, on the base handle's stream; ms[0..5]
 * receive the mean device time in milliseconds of the primal SpMM, the dual SpMM,
 * the step control, the column check, the row check and the check control (0 where
 * a kernel did not run).  The pairs move on by those attempts.
 * Errors: INVALID_ARG (null, attempts < 1), CUDA. */
int scylla_fanout_time_kernels(scylla_fanout* f, int32_t attempts, double* ms);

/* Message of the last failing call on this thread ("" if none). */
const char* scylla_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SCYLLA_H */
