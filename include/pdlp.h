/*
 * pdlp.h -- C ABI of the GB300 (sm_103a) PDLP library.
 *
 * PDLP is restarted primal-dual hybrid gradient for linear programming
 * (Applegate et al., "Practical Large-Scale Linear Programming using
 * Primal-Dual Hybrid Gradient").  The library solves
 *
 *     minimise c^T x  subject to  K_i x >= q_i   (ineq_mask[i] = 1)
 *                                 K_i x  = q_i   (ineq_mask[i] = 0)
 *                                 l <= x <= u                        (Section 2, Eq. (1))
 *
 * through the saddle problem min_{x in X} max_{y in Y} c^T x - y^T K x + q^T y
 * (Section 2, Eq. (2)) with Algorithm 1 (restarted, adaptive-step PDHG),
 * after the diagonal preconditioning of Section 3.5.  Every step of the
 * iteration runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *   - Array arguments may be HOST or DEVICE pointers (any memory the CUDA
 *     runtime can address with unified virtual addressing).  The library
 *     copies inputs in and results out with cudaMemcpyDefault on the context's
 *     stream and returns only after the results are in place.
 *   - Inputs are copied: the caller may free or reuse them when a call returns.
 *   - Dense vectors are float64, contiguous.  K is CSR: row_ptr int32[m+1]
 *     (row_ptr[0] = 0, non-decreasing), col_idx int32[nnz] (in [0, n),
 *     strictly increasing within a row: sorted, no duplicates), val
 *     float64[nnz] (finite).
 *   - Bounds may be -INFINITY (l) or +INFINITY (u); l_j <= u_j.  c and q are finite.
 *   - Return value: PDLP_OK (0) or a negative PDLP_ERR_* code; the message is
 *     available from pdlp_last_error().  No C++ exception crosses this boundary.
 *   - One context belongs to one stream; calls on one context must not overlap.
 */
#ifndef PDLP_H
#define PDLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define PDLP_OK 0
#define PDLP_ERR_INVALID_ARG (-1) /* malformed CSR, l > u, non-finite data, bad option */
#define PDLP_ERR_CUDA (-2)        /* a CUDA runtime call failed                           */
#define PDLP_ERR_OOM (-3)         /* device allocation failed                              */
#define PDLP_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up                    */
#define PDLP_ERR_STATE (-5)       /* call out of order (e.g. pdlp_grad before an unroll)  */

/* solver outcome (pdlp_result.status) */
#define PDLP_RUNNING 0
#define PDLP_OPTIMAL 1          /* Eq. (15) holds with epsilon = rel_tol            */
#define PDLP_ITER_LIMIT 2
#define PDLP_KKT_PASS_LIMIT 3   /* one pass = one product with K and one with K^T   */
#define PDLP_TIME_LIMIT 4
#define PDLP_NUMERICAL_ERROR 5  /* a step produced NaN / Inf                        */
#define PDLP_PRIMAL_INFEASIBLE 7 /* presolve: a row without free variables that 0 cannot satisfy */
#define PDLP_DUAL_INFEASIBLE 8   /* presolve: an empty column whose cost points to an infinite bound
                                    (the LP is unbounded when it is feasible)            */

/* arithmetic of the iteration */
#define PDLP_FP64 0         /* K, x, y and all reductions in float64                      */
#define PDLP_FP32 1         /* K, x, y in float32; reductions, step control in float64    */
#define PDLP_FP32_REFINE 2  /* float32 inner solves inside a float64 iterative-refinement loop */

/* ---------------------------------------------------------------- types */
typedef struct pdlp_ctx pdlp_ctx; /* opaque, owned by the library */

typedef struct {
  int32_t m, n;          /* rows (constraints), columns (variables)          */
  int64_t nnz;           /* must equal row_ptr[m]; at most 2^31 - 1           */
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
} pdlp_csr;

typedef struct {
  double rel_tol;           /* epsilon of Eq. (15) (relative = absolute), 1e-8          */
  int64_t iter_limit;       /* accepted PDHG iterations                                  */
  int64_t kkt_pass_limit;   /* step attempts (Section 4.1 "KKT passes")                  */
  double time_limit_s;      /* wall clock of one solve, checked on the device            */
  int32_t precision;        /* PDLP_FP64 | PDLP_FP32 | PDLP_FP32_REFINE                  */
  int32_t ruiz_iters;       /* Section 3.5: 10                                           */
  int32_t pock_chambolle;   /* Section 3.5: 1 = apply Pock-Chambolle alpha = 1 after Ruiz */
  int32_t eval_every;       /* Section 3: restart / termination check every 40 iterations */
  int32_t adaptive_restart; /* 1 = restart scheme of Section 3.2, 0 = never restart       */
  int32_t pw_update;        /* 1 = Algorithm 3 primal weight updates, 0 = keep omega^0    */
  double pw_smoothing;      /* Algorithm 3 theta: 0.5                                    */
  double primal_importance; /* multiplies InitializePrimalWeight (Section 3.3): 1.0       */
  double beta_suff, beta_nec, beta_art; /* Section 3.2: 0.9, 0.1, 0.5                    */
  double eps_zero;          /* Section 3.3 epsilon_zero: 1e-10                           */
  double inner_tol;         /* PDLP_FP32_REFINE: Eq. (15) tolerance of the first inner
                               solve, 1e-7 (about what float32 resolves; a solve that
                               stalls above it stops earlier); a later round that can
                               reach rel_tol uses
                               the loosest tolerance that should get there (see
                               refine.cu).  When a round divides the relative error by
                               less than 10, makes it worse, or refine_rounds is
                               reached, float64 PDLP finishes from the refined point.
                               iter_limit, kkt_pass_limit and time_limit_s bound the
                               whole solve (all rounds and the finish)                 */
  int32_t refine_rounds;    /* PDLP_FP32_REFINE: maximum outer rounds                    */
  int32_t unroll_T;         /* >0: pdlp_solve runs T unrolled steps for pdlp_grad        */
  int32_t ckpt_every;       /* unrolled steps between stored checkpoints                 */
  int32_t use_graph;        /* 1: one CUDA graph per solve (conditional WHILE nodes);
                               0: the same kernels launched from a host loop that reads
                               the state after every step attempt (for profilers)       */
  int32_t persistent;       /* step engine.  1 (default), 3, 4: all step attempts
                               between two evaluations run in one cooperative kernel
                               with grid-wide barriers (one CTA per SM); where its
                               layout does not fit, one launch per half-step.  Its
                               gathers go through L1 (after acquiring barriers) when
                               the working set of an attempt exceeds L2, else through
                               L2 only; 3 forces L2-only, 4 forces L1 gathers.  0: one
                               launch per half-step (primal, dual) over row-aligned
                               warp chunks.  2: one launch per half-step over fixed
                               256-nonzero slabs, one warp per slab (equal work per
                               warp whatever the row lengths).  pdlp_result.engine
                               reports the engine that ran.                          */
  int32_t step_policy;      /* 0 (default): Algorithm 2's adaptive step; 1: constant
                               step eta = 0.9 / ||K~||_2 with ||K~||_2 estimated by 200
                               power iterations (Section 2's baseline PDHG step); 2:
                               the Malitsky-Pock line search of Appendix C.1 (runs
                               on the per-launch engine; not with unroll_T > 0)     */
  int32_t presolve;         /* 1: presolve-lite before the solve (fixed variables l = u
                               substituted, rows left empty dropped, empty columns set
                               at the bound their cost points to); the solution and
                               Eq. (15) are reported on the original LP.  0 (default):
                               none.  Not with unroll_T > 0.                            */
  double omega0;            /* > 0: initial primal weight (Section 2's baseline PDHG
                               uses 1); 0 (default): InitializePrimalWeight          */
  int32_t restart_to_current; /* 1 (default): GetRestartCandidate of Section 3.2; 0: the
                               restart candidate is always the average (Appendix C.2,
                               "adaptive restart (theory)" with beta_suff = beta_nec =
                               0.37).  With adaptive_restart = 0 and pw_update = 1 the
                               primal weight is still updated at the evaluations where
                               the artificial criterion would restart (k = 40, 80, 160,
                               ... with the defaults; Appendix C.2 "no restart").     */
  int32_t wait_limit_us;    /* bound of every device-side wait (the grid-wide barriers of
                               the persistent step kernel), microseconds; 0 (default):
                               2 s.  A wait that runs out records the failure, the
                               kernel returns, and pdlp_solve returns PDLP_ERR_TIMEOUT
                               with the context still usable.  A negative value -N
                               bounds the waits at N us AND makes the first barrier of
                               each persistent launch wait for one arrival more than
                               the grid has, so that it always runs out: a test of
                               that path that faults and hangs nothing.              */
  double mp_breaking;       /* step_policy 2: breaking factor, 1.0 (Appendix C.1)      */
  double mp_downscaling;    /* step_policy 2: downscaling factor in (0, 1), 0.5        */
  double mp_interpolation;  /* step_policy 2: interpolation coefficient in [0, 1], 0.4 */
  void *stream;             /* cudaStream_t for all work; NULL = legacy default stream   */
} pdlp_options;

typedef struct {
  int32_t status;                 /* PDLP_OPTIMAL, ... */
  int32_t returned_average;       /* 1 if the returned point is the step-weighted average */
  int64_t iters, kkt_passes, restarts;
  int32_t refine_rounds;          /* outer rounds used by PDLP_FP32_REFINE                 */
  int32_t engine;                 /* step engine that ran the attempts: 0 warp chunks, one launch per
                                     half-step; 1 persistent warp-chunk kernel; 2 slab kernels  */
  double primal_obj, dual_obj;    /* Eq. (15) at the returned point, original problem     */
  double gap, pres, dres;         /* absolute left-hand sides of Eq. (15a-c)              */
  double rel_gap, rel_pres, rel_dres; /* each divided by its right-hand factor            */
  double seconds;                 /* device wall time of the solve                        */
  double step_size, primal_weight; /* eta and omega at the end of the solve              */
  int64_t finish_iters;           /* PDLP_FP32_REFINE: iterations of the float64 finish
                                     (counted in iters too); 0 if the float32 rounds
                                     reached rel_tol or a limit                          */
} pdlp_result;

/* ---------------------------------------------------------------- calls */

/* Fills *opts with the paper's defaults (Sections 3.1-3.5, Appendix G flags). */
int pdlp_default_options(pdlp_options *opts);

/* Builds a solver context for one LP in the form of Eq. (1).
 * Validates the data on the device, copies it, builds K^T (stable CSR
 * transpose), applies `ruiz_iters` Ruiz steps and one Pock-Chambolle step
 * (Section 3.5) to K and K^T, transforms c, q, l, u, and captures the CUDA
 * graphs of the iteration.  Returns PDLP_ERR_INVALID_ARG for malformed input
 * (nothing is allocated then).  *out receives the context.
 * With opts.presolve = 1 the reductions run first on the device and the rest
 * is built for the reduced LP (nothing when the presolve alone decides the
 * LP: solved, PDLP_PRIMAL_INFEASIBLE or PDLP_DUAL_INFEASIBLE, reported by
 * pdlp_solve).  A presolved context answers pdlp_solve, pdlp_get_trace and
 * pdlp_time_step_kernels; the calls that work in the scaled space of one LP
 * (pdlp_get_scaled, pdlp_normalized_gap, pdlp_unroll, pdlp_grad) return
 * PDLP_ERR_STATE. */
int pdlp_create(const pdlp_csr *K, const double *c, const double *q, const double *l,
                const double *u, const uint8_t *ineq_mask, const pdlp_options *opts,
                pdlp_ctx **out);

/* Runs Algorithm 1 from z^{0,0} = (x0, y0) (NULL = zero vectors, Section 4.1)
 * until Eq. (15) holds with epsilon = rel_tol or a limit is hit.  x_out (n)
 * and y_out (m) receive the returned point in the original (unscaled)
 * space: the iterate that passed the test (current first, then the average),
 * else the current iterate.  Either output may be NULL.  With
 * opts.unroll_T > 0 the call instead runs the unrolled map used by pdlp_grad
 * (see pdlp_unroll) and returns x_T, y_T. */
int pdlp_solve(pdlp_ctx *ctx, const double *x0, const double *y0, double *x_out,
               double *y_out, pdlp_result *res);

/* Unrolled PDHG for differentiation: T steps of Eq. (3) on the
 * preconditioned problem with omega = InitializePrimalWeight (fixed) and the
 * step sizes of Algorithm 2 (accepted steps), which are recorded and then
 * held constant.  Stores (x, y) every ckpt_every steps for pdlp_grad.
 * eta_out (T, nullable) receives the step sizes. */
int pdlp_unroll(pdlp_ctx *ctx, int32_t T, int32_t ckpt_every, const double *x0,
                const double *y0, double *x_out, double *y_out, double *eta_out);

/* Vector-Jacobian product of the last unrolled map (x_T, y_T) with respect
 * to (c, q, values of K): given dL/dx_T (n) and dL/dy_T (m, nullable) writes
 * dL/dc (n), dL/dq (m) and dL/dK (nnz, in the CSR order of the K passed to
 * pdlp_create).  The preconditioner and the recorded step sizes are held
 * constant; gradients accumulate in float64.  With opts.precision ==
 * PDLP_FP32 the forward map (and its recompute from the checkpoints) runs in
 * float32 and the adjoint in float64.  PDLP_ERR_STATE if no unrolled map was
 * run on ctx. */
int pdlp_grad(pdlp_ctx *ctx, const double *dL_dx, const double *dL_dy, double *dc,
              double *dq, double *dK_val);

/* Copies out the preconditioned problem built by pdlp_create (Section 3.5),
 * for inspection.  Any pointer may be NULL.  Sizes: Kval / KTval nnz
 * (float64, CSR order of K and of K^T), KT_row_ptr n+1, KT_col_idx nnz,
 * KT_perm nnz (position in K of each K^T entry), D1 m, D2 n, cs/ls/us n, qs m. */
int pdlp_get_scaled(pdlp_ctx *ctx, double *Kval, int32_t *KT_row_ptr, int32_t *KT_col_idx,
                    double *KTval, int32_t *KT_perm, double *D1, double *D2, double *cs,
                    double *qs, double *ls, double *us);

/* Section 3.2 normalized duality gap rho_r(z) on the preconditioned problem of
 * ctx, for inspection: x (n), y (m) a point of X x Y in the scaled space,
 * r > 0 the radius, omega the primal weight.  Computes K^T y and K x itself.
 * *mu receives rho_r(z), *value the maximised gap.  Float64. */
int pdlp_normalized_gap(pdlp_ctx *ctx, const double *x, const double *y, double omega,
                        double r, double *mu, double *value);

/* Batched solve of `count` independent LPs in one persistent launch (one CTA
 * per LP, largest first).  The LPs are packed back to back: LP b has
 * dims m[b], n[b]; its rows, columns and nonzeros start at row_off[b],
 * col_off[b], nnz_off[b] (int64, count+1 entries, row_off[count] = total
 * rows, ...).  row_ptr is the concatenation of the LPs' own row_ptr arrays
 * without their final entry, i.e. int32[total rows] holding offsets local to
 * each LP; col_idx (local column numbers) and val are int32 / float64[total
 * nnz]; c, l, u are float64[total cols]; q float64[total rows]; ineq_mask
 * uint8[total rows].  x_out / y_out (float64[total cols] / [total rows],
 * nullable) receive the solutions, res[count] (nullable) the outcomes.
 * Uses opts.precision (PDLP_FP64 or PDLP_FP32 arithmetic in the SpMVs, or
 * PDLP_FP32_REFINE: float32 steps until Eq. (15) holds at
 * max(rel_tol, inner_tol) or an LP stops gaining 10% in 10 evaluations, then
 * a second launch of float64 steps to rel_tol from each LP's float32 point
 * with what is left of its iteration and KKT-pass budgets; res then counts
 * both stages and refine_rounds = 1),
 * rel_tol, iter_limit, kkt_pass_limit, the preconditioner, restart, primal
 * weight and step settings, and opts.stream (step_policy must be 0 and omega0
 * 0: Algorithm 2 and InitializePrimalWeight).  Each LP needs m + n <= 4096;
 * invalid data (column index out of range or not increasing within a row,
 * non-finite value, l > u) returns PDLP_ERR_INVALID_ARG naming the first such
 * LP.  All arrays may be host or device memory. */
int pdlp_solve_batch(int32_t count, const int32_t *m, const int32_t *n, const int64_t *row_off,
                     const int64_t *col_off, const int64_t *nnz_off, const int32_t *row_ptr,
                     const int32_t *col_idx, const double *val, const double *c,
                     const double *q, const double *l, const double *u,
                     const uint8_t *ineq_mask, const pdlp_options *opts, double *x_out,
                     double *y_out, pdlp_result *res);

/* The lanes per row of K and of K^T that the batch autotuner chose for each
 * size bucket (mean row length of K: < 8, < 16, < 32, < 64, >= 64) of the
 * given precision (PDLP_FP64 or PDLP_FP32), 0 where no batch of that bucket
 * was solved yet in this process.  The autotuner times every candidate on a
 * sample of the bucket's LPs (100 steps each) the first time a bucket
 * appears and keeps the fastest.  lanes_k, lanes_kt: host int32[nbuckets]. */
int pdlp_batch_lanes(int32_t precision, int32_t *lanes_k, int32_t *lanes_kt, int32_t nbuckets);

/* Restart evaluations of the last solve on ctx, oldest first (a ring keeps
 * the last 2048).  Each record is 16 float64: k, t, mu(current), mu(average),
 * mu_0, candidate (0 current, 1 average), restarted (0/1), primal weight
 * after the evaluation (Section 3.2 and Algorithm 3), the radii
 * ||z - z^{n,0}||_omega of the current and the average iterate, and the
 * relative gap, primal and dual residuals of Eq. (15) of the current, then
 * the average iterate.  out holds 16 * max_records doubles (host or device);
 * *count receives the number of evaluations of the solve (may exceed 2048). */
int pdlp_get_trace(pdlp_ctx *ctx, double *out, int32_t max_records, int32_t *count);

/* Measures the two kernels of one step attempt of Algorithm 2 (the fused
 * K^T y product with the primal projection, and the fused K x' product with
 * the dual projection, reductions and step test) by launching each `reps`
 * times outside the solve graph on the context's stream, bracketed by CUDA
 * events.  The attempts continue from the state the last solve left (call
 * pdlp_solve first).  ms[0], ms[1] (host) receive the mean durations in
 * milliseconds of the primal and the dual kernel; ms[2] receives the mean
 * duration of one step attempt inside the persistent step kernel, timed over
 * `reps` launches of it that each run up to eval_every accepted steps (0 when
 * the context's `persistent` option is 0); ms[3] receives the mean duration
 * of one launch of the persistent evaluation kernel (the products and
 * Eq. (15) terms of one evaluation; float64 contexts with the persistent
 * step kernel, else 0), timed over `reps` launches on the state as it
 * stands.  `ms` holds 4 floats.  This call leaves the state advanced: solve
 * again before reading results. */
int pdlp_time_step_kernels(pdlp_ctx *ctx, int32_t reps, float *ms);

/* The normalized duality gap of pdlp_normalized_gap, for callers that cannot
 * allocate device memory (for example when another allocator already owns
 * the GPU's memory, or when the cost and implicit synchronisation of
 * cudaMalloc / cudaFree are not acceptable).  The paper has no counterpart of
 * this call; it allocates nothing.
 *   n, m             numbers of primal and dual coordinates, n + m <= 1048576
 *                    (larger sizes return PDLP_ERR_INVALID_ARG);
 *   x, gx, l, u      DEVICE float64[n]: point, gradient K^T y - c, bounds;
 *   y, gy, ylo       DEVICE float64[m]: point, gradient q - K x, lower bounds
 *                    of y (-INFINITY on equality rows);
 *   omega, r         primal weight and radius, both > 0;
 *   stream           cudaStream_t for the work (NULL = legacy default stream);
 *   *mu, *value      HOST outputs: rho_r(z) and the maximised gap (value nullable).
 * Scratch is one static device array of about 4.05 MiB, held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with the device
 * current) and sets the kernel's shared-memory limit; make that first call
 * before any stream capture.  Every call clears the parts of the array that
 * must start at zero; all calls share the array, so calls that overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  Returns after the result is on the host. */
int pdlp_normalized_gap_noalloc(int32_t n, int32_t m, const double *x, const double *y,
                                const double *gx, const double *gy, const double *l,
                                const double *u, const double *ylo, double omega, double r,
                                void *stream, double *mu, double *value);

/* Message of the last failing call on this thread (ctx may be NULL). */
const char *pdlp_last_error(const pdlp_ctx *ctx);

/* Frees the context and every device buffer it owns.  NULL is a no-op. */
void pdlp_destroy(pdlp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PDLP_H */
