/* Plain FP64 CPU restatement of PDLP (Applegate et al., "Practical Large-Scale
 * Linear Programming using Primal-Dual Hybrid Gradient").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the GPU path is checked
 * against: slow, single-threaded, obviously correct loops in the order the
 * paper states them.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may call it; the GPU library neither links nor includes it, and it
 * shares no code with the GPU library.
 *
 * Problem (Section 2, Eq. (1)): minimise c^T x  s.t.  K_i x >= q_i (ineq[i]=1),
 * K_i x = q_i (ineq[i]=0),  l <= x <= u  (l may be -inf, u may be +inf).
 * K is CSR with int32 indices, sorted columns, no duplicates.
 */
#ifndef PDLP_ORACLE_H
#define PDLP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_RUNNING = 0, OR_OPTIMAL = 1, OR_ITER_LIMIT = 2, OR_KKT_PASS_LIMIT = 3,
       OR_NUMERICAL_ERROR = 5 };

typedef struct {
  int32_t m, n;
  const int32_t *row_ptr, *col_idx;
  const double *val;
  const double *c, *q, *l, *u;
  const uint8_t *ineq;
  const double *ylo;  /* nullable.  Lower bound of y_i on inequality rows; NULL
                         means 0 (the paper's Y).  Equality rows are free.
                         Only the refinement correction problems set it. */
} or_lp;

typedef struct {
  double eps;              /* Eq. (15) tolerance (relative = absolute)          */
  int64_t iter_limit;      /* accepted iterations                                */
  int64_t kkt_pass_limit;  /* one K and one K^T product per step attempt         */
  int32_t ruiz_iters;      /* Section 3.5: 10                                    */
  int32_t pock_chambolle;  /* Section 3.5: 1 -> apply alpha = 1 after Ruiz       */
  double pw_theta;         /* Algorithm 3 smoothing: 0.5                         */
  double beta_suff, beta_nec, beta_art;  /* Section 3.2: 0.9, 0.1, 0.5           */
  int32_t eval_every;      /* Section 3: restart / termination check every 40    */
  double eps_zero;         /* Section 3.3 epsilon_zero                           */
  int32_t adaptive_restart;/* 1: restart scheme of Section 3.2; 0: never restart
                              (Appendix C.2 "no restart": with pw_update, the
                              primal weight is still updated at the evaluations
                              where an artificial restart would have fired)     */
  int32_t pw_update;       /* 1: Algorithm 3 at restarts; 0: keep initial omega  */
  int32_t step_policy;     /* 0: Algorithm 2; 1: constant eta = 0.9 / ||K~||_2,
                              ||K~||_2 by power iteration (Section 2's baseline
                              PDHG step; the "fixed step size" ablation);
                              2: Malitsky-Pock line search (Appendix C.1)        */
  double omega0;           /* > 0: initial primal weight; 0: InitializePrimalWeight */
  int32_t restart_to_current; /* 1: GetRestartCandidate (Section 3.2); 0: the
                              restart candidate is always the average (Appendix
                              C.2 "adaptive restart (theory)")                    */
  double mp_breaking, mp_downscaling, mp_interpolation; /* Appendix C.1: 1, 0.5, 0.4 */
} or_opts;

/* Iterations of the power iteration for ||K~||_2 (both the oracle and the
 * library use this count and the start vector 1/sqrt(n)). */
#define OR_POWER_ITERS 200

typedef struct {
  int32_t status;
  int64_t iters, kkt_passes, restarts;
  double primal_obj, dual_obj, gap, pres, dres;        /* Eq. (15) left sides   */
  double rel_gap, rel_pres, rel_dres;                  /* left / right factor   */
  double omega, eta;                                   /* final primal weight, step */
  int32_t returned_average;                            /* 1 if the average passed */
} or_result;

void or_default_opts(or_opts *o);

/* ||K~||_2 of the preconditioned K (Ruiz / Pock-Chambolle settings as given)
 * by OR_POWER_ITERS steps of power iteration on K~^T K~ from v = 1/sqrt(n):
 * w = K~ v, u = K~^T w, v = u / ||u||; returns sqrt(||u||) of the last step. */
double or_power_norm(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle);

/* K^T as CSR (n rows), stable in the row index; perm[t] = position in K of
 * the t-th entry of K^T. */
void or_transpose(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci,
                  const double *v, int32_t *trp, int32_t *tci, double *tv, int32_t *perm);

/* Section 3.5: `ruiz_iters` Ruiz iterations then (optionally) one
 * Pock-Chambolle alpha=1 step, applied in place to the values of K (CSR).
 * D1 (m) and D2 (n) receive the accumulated diagonal scalings, K~ = D1 K D2. */
void or_precondition(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci,
                     double *val, int32_t ruiz_iters, int32_t pock_chambolle,
                     double *D1, double *D2);

/* Scaled data of Section 3.5: c~ = D2 c, q~ = D1 q, l~ = l / D2, u~ = u / D2. */
void or_transform(int32_t m, int32_t n, const double *D1, const double *D2,
                  const double *c, const double *q, const double *l, const double *u,
                  double *cs, double *qs, double *ls, double *us);

/* Eq. (15) on the problem `lp` at (x, y); lambda = proj_Lambda(c - K^T y).
 * out[0..7] = primal_obj, dual_obj, gap, pres, dres, rel_gap, rel_pres, rel_dres. */
void or_kkt(const or_lp *lp, const double *x, const double *y, double *out);

/* Section 3.2 normalized duality gap rho_r(z) for the saddle problem Eq. (2):
 * (1/r) max { (K^T y - c)^T dx + (q - K x)^T dy : ||d||_omega <= r, z + d in Z }.
 * gx = K^T y - c (n), gy = q - K x (m).  Solved exactly by sorting the
 * breakpoints.  ylo (m) is the lower bound of y (-inf on equality rows).
 * Returns +inf when r == 0.  *value (nullable) = the maximum. */
double or_normalized_gap(int32_t n, int32_t m, const double *x, const double *y,
                         const double *gx, const double *gy, const double *l,
                         const double *u, const double *ylo, double omega, double r,
                         double *value);

/* Algorithm 2's step sizes for one attempt at step size eta after k accepted
 * steps: *eta_bar = (omega dx2 + dy2 / omega) / (2 |inter|) (+inf for a zero
 * denominator), *eta_next = min((1 - (k+2)^-0.3) eta_bar, (1 + (k+2)^-0.6) eta)
 * (the step being taken is number k + 1).  dx2 = ||x'-x||^2, dy2 = ||y'-y||^2,
 * inter = (y'-y)^T K (x'-x).  The solver accepts the attempt iff eta <= eta_bar. */
void or_step_sizes(double omega, double dx2, double dy2, double inter, double eta, int64_t k,
                   double *eta_bar, double *eta_next);

/* Algorithm 3: the new primal weight from Delta_x, Delta_y (2-norm distances
 * between consecutive restart points) and the smoothing theta. */
double or_primal_weight(double omega, double Dx, double Dy, double theta, double eps_zero);

/* Section 3.2 restart criteria: 1 (i), 2 (ii), 3 (iii) or 0 (no restart). */
int32_t or_restart_check(double muc, double mu0, double muc_prev, int64_t t, int64_t k,
                         double beta_suff, double beta_nec, double beta_art);

/* Algorithm 1 with Algorithm 2 steps, Section 3.2 restarts and Algorithm 3
 * primal weights, after the Section 3.5 preconditioning.  x0, y0 nullable
 * (zero start).  Outputs are in the original space. */
void or_solve(const or_lp *lp, const or_opts *opts, const double *x0, const double *y0,
              double *x_out, double *y_out, or_result *res);

/* or_solve that also records each restart evaluation (up to trace_cap) as
 * OR_TRACE_LEN doubles: k, t, mu_current, mu_average, mu_0, candidate (0
 * current, 1 average), restarted (0/1; 2 = the no-restart mode's primal
 * weight update, with mu_*, mu_0 and the radii NaN), primal weight after the
 * evaluation, the radii ||z - z^{n,0}||_omega of the current and the average
 * iterate, then the relative Eq. (15) terms (gap, primal, dual) of the
 * current and of the average iterate on the original problem.
 * *trace_n receives the number of evaluations. */
#define OR_TRACE_LEN 16
void or_solve_traced(const or_lp *lp, const or_opts *opts, const double *x0, const double *y0,
                     double *x_out, double *y_out, or_result *res, double *trace, int32_t trace_cap,
                     int32_t *trace_n);

/* Plain PDHG of Eq. (3) with constant eta and omega on the unscaled problem
 * (Appendix A): T steps from (x, y) in place. */
void or_pdhg_fixed(const or_lp *lp, double eta, double omega, int64_t T,
                   double *x, double *y);

/* Unrolled PDHG on the preconditioned problem.  The preconditioner D1, D2
 * comes from or_precondition with the given Ruiz / PC settings and is held
 * fixed; omega = InitializePrimalWeight of the scaled data (fixed).
 * Step sizes follow Algorithm 2 (accepted steps only); they are recorded in
 * eta_out[T] and treated as constants by the two functions below. */
void or_unroll_schedule(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                        int64_t T, const double *x0, const double *y0,
                        double *eta_out, double *omega_out, double *x_out, double *y_out);

/* Forward map with a given schedule: T steps of Eq. (3) (tau = eta/omega,
 * sigma = eta*omega) on the scaled problem, returning x_T, y_T in the
 * original space. */
void or_unroll_forward(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                       int64_t T, const double *eta, double omega, const double *x0,
                       const double *y0, double *x_out, double *y_out);

/* Vector-Jacobian product of the forward map: given dL/dx_T (n) and dL/dy_T
 * (m, nullable) returns dL/dc (n), dL/dq (m), dL/dK (nnz, CSR order of K).
 * Plain reverse mode over all T stored iterates. */
void or_unroll_vjp(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                   int64_t T, const double *eta, double omega, const double *x0,
                   const double *y0, const double *gx_T, const double *gy_T,
                   double *dc, double *dq, double *dK);

/* Correction LP for iterative refinement at (xh, yh) (original space):
 *   c' = dD (c - K^T yh),  q' = dP (q - K xh),
 *   l' = dP (l - xh),      u' = dP (u - xh),
 *   y lower bound on inequality rows = -dD * yh  (written as ylo', -inf on equality rows)
 * with dP = 1 / max(primal violation inf-norm, tiny), dD = 1 / max(dual
 * violation inf-norm, tiny), each clipped to [1, dmax].  A saddle point
 * (a, b) of the correction problem gives x = xh + a/dP, y = yh + b/dD. */
void or_correction_lp(const or_lp *lp, const double *xh, const double *yh, double dmax,
                      double *cp, double *qp, double *lp_, double *up, double *ylo,
                      double *dP, double *dD);

#ifdef __cplusplus
}
#endif
#endif
