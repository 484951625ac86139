/* Plain FP64 CPU restatement of PDLP -- TEST INFRASTRUCTURE ONLY.
 *
 * Every function follows the paper's statement directly (sections, equations
 * and algorithms are cited at each function).  Loops are sequential and in
 * index order; there is no blocking, fusion or reordering.  Built with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Readings of the paper taken where it is silent or ambiguous (each one is
 * listed with its justification in the design notes of the repository):
 *  R1  dual objective  q^T y + sum_j l_j max(lambda_j,0) + u_j min(lambda_j,0)
 *      (Eq. (1) writes -u^T lambda^- with lambda^- = min(0, lambda); weak
 *      duality fixes the sign to +)
 *  R3  diagonal preconditioning divides by the square roots of the norms:
 *      K~_ij = (K_ij / sqrt(r_i)) / sqrt(s_j), zero norms give a factor 1
 *  R4  ||K||_inf in Algorithm 1's initial step is max_ij |K~_ij|
 *  R5  Algorithm 2's denominator is 2|(y'-y)^T K (x'-x)| (its magnitude: then
 *      eta_bar >= 1/||K||_2 holds always, as Section 3.1 states); zero gives
 *      eta_bar = +inf
 *  R6  mu_0 = +inf in the first outer loop; "previous candidate" mu is the
 *      one of the previous evaluation in the same outer loop (+inf at first)
 *  R7  r = 0 gives mu = +inf
 *  R8  epsilon_zero = 1e-10
 *  R9  termination is tested on the original problem, current iterate first,
 *      then the average
 *  R10 every step attempt costs one KKT pass
 *  R11 Algorithm 2's k is the 1-based number of the step being taken (Algorithm
 *      1's counter plus one), so the first step uses (1 - 2^-0.3)
 *  R12 the normalized gap is defined for z in Z; the step-weighted average can
 *      leave its box by an ulp after rounding, so distances to the bounds are
 *      taken as max(distance, 0)
 */
#include "pdlp_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ORACLE_TRACE=1 in the environment prints one line per restart evaluation,
 * ORACLE_TRACE=2 also one line per step attempt. */
static int trace_on(void) {
  static int on = -1;
  if (on < 0) { const char *e = getenv("ORACLE_TRACE"); on = e ? atoi(e) : 0; }
  return on;
}

static double *dalloc(size_t n) {
  double *p = (double *)calloc(n ? n : 1, sizeof(double));
  if (!p) abort();
  return p;
}
static int32_t *ialloc(size_t n) {
  int32_t *p = (int32_t *)calloc(n ? n : 1, sizeof(int32_t));
  if (!p) abort();
  return p;
}

void or_default_opts(or_opts *o) {
  o->eps = 1e-8;
  o->iter_limit = 1000000;
  o->kkt_pass_limit = 4000000;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->pw_theta = 0.5;
  o->beta_suff = 0.9;
  o->beta_nec = 0.1;
  o->beta_art = 0.5;
  o->eval_every = 40;
  o->eps_zero = 1e-10;
  o->adaptive_restart = 1;
  o->pw_update = 1;
  o->step_policy = 0;
  o->omega0 = 0.0;
  o->restart_to_current = 1;
  o->mp_breaking = 1.0;
  o->mp_downscaling = 0.5;
  o->mp_interpolation = 0.4;
}

/* ---------------------------------------------------------------- basics */

/* y = K x for CSR K */
static void spmv(int32_t m, const int32_t *rp, const int32_t *ci, const double *v,
                 const double *x, double *y) {
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
    y[i] = s;
  }
}

/* y = K^T x computed from K's rows: column sums accumulate in row order. */
static void spmv_t(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci,
                   const double *v, const double *x, double *y) {
  for (int32_t j = 0; j < n; ++j) y[j] = 0.0;
  for (int32_t i = 0; i < m; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) y[ci[k]] += v[k] * x[i];
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
static double norm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

static double clip(double v, double lo, double hi) {
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

/* lower bound of y_i: the paper's Y (0 on inequality rows, free on equality rows)
 * unless the problem carries its own */
static double ylo_of(const or_lp *lp, int32_t i) {
  if (!lp->ineq[i]) return -INFINITY;
  return lp->ylo ? lp->ylo[i] : 0.0;
}

/* ------------------------------------------------------------- transpose */

void or_transpose(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci,
                  const double *v, int32_t *trp, int32_t *tci, double *tv, int32_t *perm) {
  for (int32_t j = 0; j <= n; ++j) trp[j] = 0;
  for (int32_t k = 0; k < rp[m]; ++k) trp[ci[k] + 1] += 1;
  for (int32_t j = 0; j < n; ++j) trp[j + 1] += trp[j];
  int32_t *next = ialloc((size_t)n);
  for (int32_t j = 0; j < n; ++j) next[j] = trp[j];
  for (int32_t i = 0; i < m; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      int32_t t = next[ci[k]]++;
      tci[t] = i;
      if (tv) tv[t] = v[k];
      if (perm) perm[t] = k;
    }
  free(next);
}

/* ------------------------------------------------------- Section 3.5 */

/* One rescaling step: r (m) and s (n) hold the row / column norms of the
 * current K~; divide by their square roots (R3). */
static void rescale(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, double *val,
                    double *r, double *s, double *D1, double *D2) {
  for (int32_t i = 0; i < m; ++i) r[i] = r[i] > 0.0 ? sqrt(r[i]) : 1.0;
  for (int32_t j = 0; j < n; ++j) s[j] = s[j] > 0.0 ? sqrt(s[j]) : 1.0;
  for (int32_t i = 0; i < m; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) val[k] = val[k] / r[i] / s[ci[k]];
  for (int32_t i = 0; i < m; ++i) D1[i] = D1[i] / r[i];
  for (int32_t j = 0; j < n; ++j) D2[j] = D2[j] / s[j];
}

void or_precondition(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci,
                     double *val, int32_t ruiz_iters, int32_t pock_chambolle,
                     double *D1, double *D2) {
  double *r = dalloc((size_t)m), *s = dalloc((size_t)n);
  for (int32_t i = 0; i < m; ++i) D1[i] = 1.0;
  for (int32_t j = 0; j < n; ++j) D2[j] = 1.0;
  /* Ruiz: row and column infinity norms of the current matrix */
  for (int32_t it = 0; it < ruiz_iters; ++it) {
    for (int32_t i = 0; i < m; ++i) r[i] = 0.0;
    for (int32_t j = 0; j < n; ++j) s[j] = 0.0;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        double a = fabs(val[k]);
        if (a > r[i]) r[i] = a;
        if (a > s[ci[k]]) s[ci[k]] = a;
      }
    rescale(m, n, rp, ci, val, r, s, D1, D2);
  }
  /* Pock-Chambolle with alpha = 1: row norm ||.||_{2-alpha} = l1, column ||.||_alpha = l1 */
  if (pock_chambolle) {
    for (int32_t i = 0; i < m; ++i) r[i] = 0.0;
    for (int32_t j = 0; j < n; ++j) s[j] = 0.0;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        double a = fabs(val[k]);
        r[i] += a;
        s[ci[k]] += a;
      }
    rescale(m, n, rp, ci, val, r, s, D1, D2);
  }
  free(r);
  free(s);
}

void or_transform(int32_t m, int32_t n, const double *D1, const double *D2,
                  const double *c, const double *q, const double *l, const double *u,
                  double *cs, double *qs, double *ls, double *us) {
  for (int32_t j = 0; j < n; ++j) {
    cs[j] = D2[j] * c[j];
    ls[j] = l[j] / D2[j];
    us[j] = u[j] / D2[j];
  }
  for (int32_t i = 0; i < m; ++i) qs[i] = D1[i] * q[i];
}

/* ------------------------------------------------------------ Eq. (15) */

void or_kkt(const or_lp *lp, const double *x, const double *y, double *out) {
  int32_t m = lp->m, n = lp->n;
  double *Kx = dalloc((size_t)m), *KTy = dalloc((size_t)n);
  spmv(m, lp->row_ptr, lp->col_idx, lp->val, x, Kx);
  spmv_t(m, n, lp->row_ptr, lp->col_idx, lp->val, y, KTy);
  double pobj = dot(n, lp->c, x);
  double pres2 = 0.0, dres2 = 0.0, dobj = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    double r = lp->q[i] - Kx[i];
    if (lp->ineq[i]) {
      double lo = ylo_of(lp, i);
      if (lo != 0.0 && lo > -INFINITY) pobj += lo * r; /* only for a general dual bound */
      r = r > 0.0 ? r : 0.0;                           /* (h - Gx)^+ */
    }
    pres2 += r * r;
    dobj += lp->q[i] * y[i];
  }
  for (int32_t j = 0; j < n; ++j) {
    double rc = lp->c[j] - KTy[j];
    int lf = isfinite(lp->l[j]), uf = isfinite(lp->u[j]);
    double lam; /* proj_Lambda, Lambda_j from the finiteness of l_j, u_j (Section 2) */
    if (!lf && !uf) lam = 0.0;
    else if (!lf) lam = rc < 0.0 ? rc : 0.0;
    else if (!uf) lam = rc > 0.0 ? rc : 0.0;
    else lam = rc;
    dres2 += (rc - lam) * (rc - lam);
    if (lam > 0.0) dobj += lp->l[j] * lam; /* R1 */
    if (lam < 0.0) dobj += lp->u[j] * lam;
  }
  double gap = fabs(dobj - pobj);
  double pres = sqrt(pres2), dres = sqrt(dres2);
  out[0] = pobj;
  out[1] = dobj;
  out[2] = gap;
  out[3] = pres;
  out[4] = dres;
  out[5] = gap / (1.0 + fabs(dobj) + fabs(pobj));
  out[6] = pres / (1.0 + norm2(m, lp->q));
  out[7] = dres / (1.0 + norm2(n, lp->c));
  free(Kx);
  free(KTy);
}

/* ------------------------------------------- Section 3.2 normalized gap */

typedef struct { double t, a, w, v; } gap_item;

static int cmp_item(const void *pa, const void *pb) {
  double ta = ((const gap_item *)pa)->t, tb = ((const gap_item *)pb)->t;
  return (ta > tb) - (ta < tb);
}

/* The maximiser of g^T d over {||d||_omega <= r} intersected with the box
 * z + d in Z is d(t) = (clip(t gx/omega, l-x, u-x), clip(t omega gy, ylo-y, +inf))
 * for the t >= 0 at which ||d(t)||_omega = r (t = +inf if the whole box corner
 * lies inside the ball).  Coordinate i stays unclipped up to its breakpoint
 * t_i; phi(t) = ||d(t)||^2_omega = sum_{t_i <= t} w_i + t^2 sum_{t_i > t} a_i
 * and g^T d(t) = sum_{t_i <= t} v_i + t sum_{t_i > t} a_i.  The items are
 * sorted by t_i and the crossing segment is solved in closed form. */
double or_normalized_gap(int32_t n, int32_t m, const double *x, const double *y,
                         const double *gx, const double *gy, const double *l,
                         const double *u, const double *ylo, double omega, double r,
                         double *value) {
  if (value) *value = 0.0;
  if (!(r > 0.0)) return INFINITY; /* R7 */
  gap_item *it = (gap_item *)malloc(sizeof(gap_item) * ((size_t)n + (size_t)m + 1));
  if (!it) abort();
  int64_t cnt = 0;
  for (int32_t j = 0; j < n; ++j) {
    double g = gx[j];
    if (g == 0.0) continue;
    double dist = g > 0.0 ? u[j] - x[j] : x[j] - l[j];
    if (!(dist > 0.0)) dist = 0.0; /* R12 */
    double ag = fabs(g);
    gap_item e;
    e.a = g * g / omega;
    if (isinf(dist)) { e.t = INFINITY; e.w = 0.0; e.v = 0.0; }
    else { e.t = omega * dist / ag; e.w = omega * dist * dist; e.v = ag * dist; }
    it[cnt++] = e;
  }
  for (int32_t i = 0; i < m; ++i) {
    double g = gy[i];
    if (g == 0.0) continue;
    double dist = g > 0.0 ? INFINITY : y[i] - ylo[i];
    if (!(dist > 0.0)) dist = 0.0; /* R12 */
    double ag = fabs(g);
    gap_item e;
    e.a = omega * g * g;
    if (isinf(dist)) { e.t = INFINITY; e.w = 0.0; e.v = 0.0; }
    else { e.t = dist / (omega * ag); e.w = dist * dist / omega; e.v = ag * dist; }
    it[cnt++] = e;
  }
  qsort(it, (size_t)cnt, sizeof(gap_item), cmp_item);
  double *suffix = dalloc((size_t)cnt + 1); /* suffix[k] = sum_{i >= k} a_i */
  suffix[cnt] = 0.0;
  for (int64_t k = cnt - 1; k >= 0; --k) suffix[k] = suffix[k + 1] + it[k].a;
  double target = r * r, W = 0.0, V = 0.0, best;
  int64_t k = 0;
  for (; k < cnt && isfinite(it[k].t); ++k) {
    double phi = W + it[k].t * it[k].t * suffix[k];
    if (phi >= target) break;
    W += it[k].w;
    V += it[k].v;
  }
  double A = suffix[k];
  if (A > 0.0) {
    double t = sqrt((target - W) / A);
    best = V + t * A;
  } else {
    best = V; /* every coordinate reached its bound inside the ball */
  }
  free(it);
  free(suffix);
  if (value) *value = best;
  return best / r;
}

/* --------------------------------------------------- Algorithms 1, 2, 3 */

/* Everything the iteration needs on the preconditioned problem. */
typedef struct {
  int32_t m, n;
  const int32_t *rp, *ci;
  double *v;              /* K~ values (CSR of K)   */
  int32_t *trp, *tci;
  double *tv;             /* K~^T values            */
  double *c, *q, *l, *u, *ylo;  /* scaled data       */
  double *D1, *D2;
} scaled_lp;

static void scaled_build(const or_lp *lp, int32_t ruiz, int32_t pc, scaled_lp *s) {
  int32_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
  s->m = m;
  s->n = n;
  s->rp = lp->row_ptr;
  s->ci = lp->col_idx;
  s->v = dalloc((size_t)nnz);
  memcpy(s->v, lp->val, sizeof(double) * (size_t)nnz);
  s->D1 = dalloc((size_t)m);
  s->D2 = dalloc((size_t)n);
  or_precondition(m, n, lp->row_ptr, lp->col_idx, s->v, ruiz, pc, s->D1, s->D2);
  s->trp = ialloc((size_t)n + 1);
  s->tci = ialloc((size_t)nnz);
  s->tv = dalloc((size_t)nnz);
  or_transpose(m, n, lp->row_ptr, lp->col_idx, s->v, s->trp, s->tci, s->tv, NULL);
  s->c = dalloc((size_t)n);
  s->q = dalloc((size_t)m);
  s->l = dalloc((size_t)n);
  s->u = dalloc((size_t)n);
  s->ylo = dalloc((size_t)m);
  or_transform(m, n, s->D1, s->D2, lp->c, lp->q, lp->l, lp->u, s->c, s->q, s->l, s->u);
  for (int32_t i = 0; i < m; ++i) s->ylo[i] = ylo_of(lp, i) / s->D1[i];
}

static void scaled_free(scaled_lp *s) {
  free(s->v); free(s->D1); free(s->D2); free(s->trp); free(s->tci); free(s->tv);
  free(s->c); free(s->q); free(s->l); free(s->u); free(s->ylo);
}

static void K_mul(const scaled_lp *s, const double *x, double *out) {
  spmv(s->m, s->rp, s->ci, s->v, x, out);
}
static void KT_mul(const scaled_lp *s, const double *y, double *out) {
  spmv(s->n, s->trp, s->tci, s->tv, y, out);
}

/* ||K~||_2 by power iteration on K~^T K~ (Section 2: baseline step size) */
static double power_norm(const scaled_lp *s) {
  int32_t m = s->m, n = s->n;
  double *v = dalloc((size_t)n), *w = dalloc((size_t)m), *u = dalloc((size_t)n);
  for (int32_t j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
  double nu = 0.0;
  for (int it = 0; it < OR_POWER_ITERS; ++it) {
    K_mul(s, v, w);
    KT_mul(s, w, u);
    nu = norm2(n, u);
    if (!(nu > 0.0)) break;
    for (int32_t j = 0; j < n; ++j) v[j] = u[j] / nu;
  }
  free(v); free(w); free(u);
  return sqrt(nu);
}

double or_power_norm(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle) {
  scaled_lp s;
  scaled_build(lp, ruiz_iters, pock_chambolle, &s);
  double r = power_norm(&s);
  scaled_free(&s);
  return r;
}

/* InitializePrimalWeight (Section 3.3) */
static double init_primal_weight(const scaled_lp *s, double eps_zero) {
  double nc = norm2(s->n, s->c), nq = norm2(s->m, s->q);
  if (nc > eps_zero && nq > eps_zero) return nc / nq;
  return 1.0;
}

/* ||(dx, dy)||_omega^2 */
static double wnorm2(double omega, double dx2, double dy2) { return omega * dx2 + dy2 / omega; }

/* Algorithm 2's two step sizes for an attempt at step size eta, with k
 * accepted steps taken before it:
 *   eta_bar = ||z' - z||_omega^2 / (2 |(y' - y)^T K (x' - x)|)   (R5; a zero
 *             denominator gives +inf),
 *   eta'    = min((1 - (k' + 1)^-0.3) eta_bar, (1 + (k' + 1)^-0.6) eta)
 * with k' = k + 1 the number of the step being taken (R11). */
void or_step_sizes(double omega, double dx2, double dy2, double inter, double eta, int64_t k,
                   double *eta_bar, double *eta_next) {
  double num = wnorm2(omega, dx2, dy2);
  double den = 2.0 * fabs(inter);                           /* R5 */
  double eb = den > 0.0 ? num / den : INFINITY;
  double kk = (double)(k + 1);                              /* R11 */
  double e1 = (1.0 - pow(kk + 1.0, -0.3)) * eb;
  double e2 = (1.0 + pow(kk + 1.0, -0.6)) * eta;
  *eta_bar = eb;
  *eta_next = e1 < e2 ? e1 : e2;
}

/* Algorithm 3 (PrimalWeightUpdate): with Delta_x = ||x^{n,0} - x^{n-1,0}||_2
 * and Delta_y likewise, omega <- exp(theta log(Delta_y / Delta_x) +
 * (1 - theta) log(omega)) when both exceed epsilon_zero, else unchanged. */
double or_primal_weight(double omega, double Dx, double Dy, double theta, double eps_zero) {
  if (Dx > eps_zero && Dy > eps_zero) return exp(theta * log(Dy / Dx) + (1.0 - theta) * log(omega));
  return omega;
}

/* Section 3.2 restart criteria at an evaluation: muc = mu of the restart
 * candidate, mu0 = mu_n(z^{n,0}, z^{n-1,0}), muc_prev = the candidate's mu at
 * the previous evaluation of this outer loop (R6), t inner and k total
 * iterations.  Returns 1 for (i) sufficient decay, 2 for (ii) necessary decay
 * without local progress, 3 for (iii) artificial restart, 0 for none (the
 * first that holds, in that order). */
int32_t or_restart_check(double muc, double mu0, double muc_prev, int64_t t, int64_t k,
                         double beta_suff, double beta_nec, double beta_art) {
  if (muc <= beta_suff * mu0) return 1;
  if (muc <= beta_nec * mu0 && muc > muc_prev) return 2;
  if ((double)t >= beta_art * (double)k) return 3;
  return 0;
}

/* One attempt of Algorithm 2's loop body at step size eta: writes x', y',
 * K x', K^T y' and returns eta_bar and the next eta'. */
typedef struct { double *x, *y, *Kx, *KTy; } iterate;

static void pdhg_attempt(const scaled_lp *s, const iterate *z, iterate *zp, double eta,
                         double omega, int64_t k, double *eta_bar, double *eta_next,
                         int *bad) {
  int32_t m = s->m, n = s->n;
  for (int32_t j = 0; j < n; ++j)
    zp->x[j] = clip(z->x[j] - (eta / omega) * (s->c[j] - z->KTy[j]), s->l[j], s->u[j]);
  K_mul(s, zp->x, zp->Kx);
  for (int32_t i = 0; i < m; ++i) {
    double v = z->y[i] + eta * omega * (s->q[i] - 2.0 * zp->Kx[i] + z->Kx[i]);
    zp->y[i] = v > s->ylo[i] ? v : s->ylo[i];
  }
  KT_mul(s, zp->y, zp->KTy);
  double dx2 = 0.0, dy2 = 0.0, inter = 0.0;
  for (int32_t j = 0; j < n; ++j) dx2 += (zp->x[j] - z->x[j]) * (zp->x[j] - z->x[j]);
  for (int32_t i = 0; i < m; ++i) {
    double dy = zp->y[i] - z->y[i];
    dy2 += dy * dy;
    inter += dy * (zp->Kx[i] - z->Kx[i]);
  }
  double num = wnorm2(omega, dx2, dy2);
  or_step_sizes(omega, dx2, dy2, inter, eta, k, eta_bar, eta_next);
  *bad = !isfinite(num) || isnan(*eta_bar) || isnan(inter);
}

/* Appendix C.1, one iteration of the Malitsky-Pock line search from z:
 * the primal step x' = proj_X(x - (eta_k / omega)(c - K^T y)) is taken once;
 * each trial picks eta_hat (first eta_k + interpolation (sqrt(1 + theta_k) - 1)
 * eta_k, then times the downscaling factor), theta_hat = eta_k / eta_hat,
 * y_hat = proj_Y(y + omega eta_hat (q - K(x' + theta_hat (x' - x)))), and
 * stops when eta_hat ||K^T (y_hat - y)|| <= breaking ||y_hat - y||.  Each trial
 * adds one to *passes (its K^T product; the K product of x' belongs to the
 * first).  Writes zp, returns the accepted eta_hat and *theta_out; *accepted
 * is 0 when *passes reached pass_cap first or a value was not finite. */
static double mp_iteration(const scaled_lp *s, const or_opts *o, const iterate *z, iterate *zp,
                           double eta_k, double theta_k, double omega, double *theta_out,
                           int64_t *passes, int64_t pass_cap, int *accepted, int *bad) {
  int32_t m = s->m, n = s->n;
  for (int32_t j = 0; j < n; ++j)
    zp->x[j] = clip(z->x[j] - (eta_k / omega) * (s->c[j] - z->KTy[j]), s->l[j], s->u[j]);
  K_mul(s, zp->x, zp->Kx);
  double eh = eta_k + o->mp_interpolation * (sqrt(1.0 + theta_k) - 1.0) * eta_k;
  double th = eta_k / eh;
  *accepted = 0;
  *bad = 0;
  for (;;) {
    for (int32_t i = 0; i < m; ++i) {
      double xbar_k = zp->Kx[i] + th * (zp->Kx[i] - z->Kx[i]); /* K (x' + th (x' - x)) */
      double v = z->y[i] + omega * eh * (s->q[i] - xbar_k);
      zp->y[i] = v > s->ylo[i] ? v : s->ylo[i];
    }
    KT_mul(s, zp->y, zp->KTy);
    *passes += 1;
    double dy2 = 0.0, dk2 = 0.0;
    for (int32_t i = 0; i < m; ++i) dy2 += (zp->y[i] - z->y[i]) * (zp->y[i] - z->y[i]);
    for (int32_t j = 0; j < n; ++j) dk2 += (zp->KTy[j] - z->KTy[j]) * (zp->KTy[j] - z->KTy[j]);
    if (!isfinite(dy2) || !isfinite(dk2) || !isfinite(eh)) { *bad = 1; break; }
    if (eh * sqrt(dk2) <= o->mp_breaking * sqrt(dy2)) { *accepted = 1; break; }
    if (*passes >= pass_cap) break;
    eh *= o->mp_downscaling;
    th = eta_k / eh;
  }
  *theta_out = th;
  return eh;
}

static void copy_iterate(const scaled_lp *s, iterate *dst, const iterate *src) {
  memcpy(dst->x, src->x, sizeof(double) * (size_t)s->n);
  memcpy(dst->y, src->y, sizeof(double) * (size_t)s->m);
  memcpy(dst->Kx, src->Kx, sizeof(double) * (size_t)s->m);
  memcpy(dst->KTy, src->KTy, sizeof(double) * (size_t)s->n);
}

static void alloc_iterate(const scaled_lp *s, iterate *z) {
  z->x = dalloc((size_t)s->n);
  z->y = dalloc((size_t)s->m);
  z->Kx = dalloc((size_t)s->m);
  z->KTy = dalloc((size_t)s->n);
}
static void free_iterate(iterate *z) { free(z->x); free(z->y); free(z->Kx); free(z->KTy); }

/* mu_n(z, z_ref): normalized gap at z with radius r = ||z - z_ref||_omega
 * (*r_out, nullable, receives r) */
static double mu_of(const scaled_lp *s, const iterate *z, const double *xr, const double *yr,
                    double omega, double *r_out) {
  int32_t m = s->m, n = s->n;
  double dx2 = 0.0, dy2 = 0.0;
  for (int32_t j = 0; j < n; ++j) dx2 += (z->x[j] - xr[j]) * (z->x[j] - xr[j]);
  for (int32_t i = 0; i < m; ++i) dy2 += (z->y[i] - yr[i]) * (z->y[i] - yr[i]);
  double r = sqrt(wnorm2(omega, dx2, dy2));
  if (r_out) *r_out = r;
  double *gx = dalloc((size_t)n), *gy = dalloc((size_t)m);
  for (int32_t j = 0; j < n; ++j) gx[j] = z->KTy[j] - s->c[j];
  for (int32_t i = 0; i < m; ++i) gy[i] = s->q[i] - z->Kx[i];
  double mu = or_normalized_gap(n, m, z->x, z->y, gx, gy, s->l, s->u, s->ylo, omega, r, NULL);
  free(gx);
  free(gy);
  return mu;
}

/* Eq. (15) on the original problem at the unscaled point (R9) */
static int terminated(const or_lp *lp, const scaled_lp *s, const iterate *z, double eps,
                      double *kkt_out, double *xo, double *yo) {
  for (int32_t j = 0; j < s->n; ++j) xo[j] = s->D2[j] * z->x[j];
  for (int32_t i = 0; i < s->m; ++i) yo[i] = s->D1[i] * z->y[i];
  or_kkt(lp, xo, yo, kkt_out);
  return kkt_out[5] <= eps && kkt_out[6] <= eps && kkt_out[7] <= eps;
}

static void fill_result(or_result *res, const double *kkt) {
  res->primal_obj = kkt[0];
  res->dual_obj = kkt[1];
  res->gap = kkt[2];
  res->pres = kkt[3];
  res->dres = kkt[4];
  res->rel_gap = kkt[5];
  res->rel_pres = kkt[6];
  res->rel_dres = kkt[7];
}

void or_solve(const or_lp *lp, const or_opts *o, const double *x0, const double *y0,
              double *x_out, double *y_out, or_result *res) {
  or_solve_traced(lp, o, x0, y0, x_out, y_out, res, NULL, 0, NULL);
}

void or_solve_traced(const or_lp *lp, const or_opts *o, const double *x0, const double *y0,
                     double *x_out, double *y_out, or_result *res, double *trace, int32_t trace_cap,
                     int32_t *trace_n) {
  int32_t ntr = 0;
  memset(res, 0, sizeof(*res));
  scaled_lp s;
  scaled_build(lp, o->ruiz_iters, o->pock_chambolle, &s);
  int32_t m = s.m, n = s.n, nnz = lp->row_ptr[m];
  iterate z, zp, zbar;
  alloc_iterate(&s, &z);
  alloc_iterate(&s, &zp);
  alloc_iterate(&s, &zbar);
  double *sx = dalloc((size_t)n), *sy = dalloc((size_t)m);   /* sum eta_i z_i */
  double *x0r = dalloc((size_t)n), *y0r = dalloc((size_t)m); /* z^{n,0}       */
  double *xo = dalloc((size_t)n), *yo = dalloc((size_t)m), kkt[8];

  /* initial point z^{0,0} (zero unless given), inside X x Y */
  for (int32_t j = 0; j < n; ++j) z.x[j] = clip(x0 ? x0[j] / s.D2[j] : 0.0, s.l[j], s.u[j]);
  for (int32_t i = 0; i < m; ++i) {
    double v = y0 ? y0[i] / s.D1[i] : 0.0;
    z.y[i] = v > s.ylo[i] ? v : s.ylo[i];
  }
  K_mul(&s, z.x, z.Kx);
  KT_mul(&s, z.y, z.KTy);

  /* Algorithm 1 initialisation */
  double kmax = 0.0;
  for (int32_t k = 0; k < nnz; ++k) kmax = fabs(s.v[k]) > kmax ? fabs(s.v[k]) : kmax;
  double eta_hat = kmax > 0.0 ? 1.0 / kmax : 1.0; /* R4 */
  if (o->step_policy == 1) {                        /* constant step 0.9 / ||K~||_2 */
    double kn = power_norm(&s);
    eta_hat = kn > 0.0 ? 0.9 / kn : 1.0;
  }
  double omega = o->omega0 > 0.0 ? o->omega0 : init_primal_weight(&s, o->eps_zero);
  int64_t k = 0, kkt_passes = 0, restarts = 0;
  int status = OR_RUNNING, ret_avg = 0;
  const iterate *ret = &z;

  if (terminated(lp, &s, &z, o->eps, kkt, xo, yo)) status = OR_OPTIMAL; /* check at start */

  memcpy(x0r, z.x, sizeof(double) * (size_t)n);
  memcpy(y0r, z.y, sizeof(double) * (size_t)m);
  double mu0 = INFINITY; /* R6 */
  double mp_theta = 1.0; /* Appendix C.1 theta_0 (R22) */
  int64_t k_virt = 0;    /* no-restart mode: iteration of the last primal weight update */

  while (status == OR_RUNNING) {            /* outer loop */
    int64_t t = 0;
    double sum_eta = 0.0, muc_prev = INFINITY;
    for (int32_t j = 0; j < n; ++j) sx[j] = 0.0;
    for (int32_t i = 0; i < m; ++i) sy[i] = 0.0;
    int restart = 0;
    while (!restart && status == OR_RUNNING) { /* inner loop */
      /* Algorithm 2 */
      double eta = eta_hat, eta_bar, eta_next;
      int bad = 0;
      if (o->step_policy == 2) { /* Appendix C.1 */
        int accepted = 0;
        double th = 1.0;
        eta = mp_iteration(&s, o, &z, &zp, eta_hat, mp_theta, omega, &th, &kkt_passes, o->kkt_pass_limit,
                           &accepted, &bad);
        if (bad) status = OR_NUMERICAL_ERROR;
        else if (!accepted) status = OR_KKT_PASS_LIMIT;
        mp_theta = th;
        eta_next = eta;
      } else for (;;) {
        pdhg_attempt(&s, &z, &zp, eta, omega, k, &eta_bar, &eta_next, &bad);
        kkt_passes += 1; /* R10 */
        if (bad) { status = OR_NUMERICAL_ERROR; break; }
        if (trace_on() > 1)
          fprintf(stderr, "  attempt k=%lld eta=%.17g eta_bar=%.17g %s\n", (long long)k, eta, eta_bar,
                  eta <= eta_bar ? "accept" : "reject");
        if (o->step_policy == 1) { eta_next = eta; break; } /* constant step: always accept */
        if (eta <= eta_bar) break;
        eta = eta_next;
        if (kkt_passes >= o->kkt_pass_limit) { status = OR_KKT_PASS_LIMIT; break; }
      }
      if (status != OR_RUNNING) break;
      eta_hat = eta_next;
      copy_iterate(&s, &z, &zp);
      /* running average with weights eta (Algorithm 1) */
      for (int32_t j = 0; j < n; ++j) sx[j] += eta * z.x[j];
      for (int32_t i = 0; i < m; ++i) sy[i] += eta * z.y[i];
      sum_eta += eta;
      t += 1;
      k += 1;
      if (k % o->eval_every != 0 && k < o->iter_limit && kkt_passes < o->kkt_pass_limit)
        continue;

      /* restart / termination evaluation (every eval_every iterations) */
      for (int32_t j = 0; j < n; ++j) zbar.x[j] = sx[j] / sum_eta;
      for (int32_t i = 0; i < m; ++i) zbar.y[i] = sy[i] / sum_eta;
      K_mul(&s, zbar.x, zbar.Kx);
      KT_mul(&s, zbar.y, zbar.KTy);
      double kc[8], ka[8]; /* Eq. (15) at the current and the average iterate */
      if (terminated(lp, &s, &z, o->eps, kc, xo, yo)) { status = OR_OPTIMAL; ret = &z; break; }
      if (terminated(lp, &s, &zbar, o->eps, ka, xo, yo)) {
        status = OR_OPTIMAL; ret = &zbar; ret_avg = 1; break;
      }
      if (k >= o->iter_limit) { status = OR_ITER_LIMIT; break; }
      if (kkt_passes >= o->kkt_pass_limit) { status = OR_KKT_PASS_LIMIT; break; }
      if (!o->adaptive_restart) {
        /* Appendix C.2 "no restart": the primal weight is still updated where
         * the artificial criterion (iii) would have restarted, measured from
         * the point of the previous update (R23) */
        if (o->pw_update && (double)(k - k_virt) >= o->beta_art * (double)k) {
          double dx2 = 0.0, dy2 = 0.0;
          for (int32_t j = 0; j < n; ++j) dx2 += (z.x[j] - x0r[j]) * (z.x[j] - x0r[j]);
          for (int32_t i = 0; i < m; ++i) dy2 += (z.y[i] - y0r[i]) * (z.y[i] - y0r[i]);
          double Dx = sqrt(dx2), Dy = sqrt(dy2);
          omega = or_primal_weight(omega, Dx, Dy, o->pw_theta, o->eps_zero);
          memcpy(x0r, z.x, sizeof(double) * (size_t)n);
          memcpy(y0r, z.y, sizeof(double) * (size_t)m);
          k_virt = k;
          if (trace && ntr < trace_cap) {
            double *rec = trace + (size_t)ntr * OR_TRACE_LEN;
            rec[0] = (double)k;
            rec[1] = (double)t;
            rec[2] = rec[3] = rec[4] = NAN;
            rec[5] = 0.0;
            rec[6] = 2.0;
            rec[7] = omega;
            rec[8] = rec[9] = NAN;
            for (int a = 0; a < 3; ++a) { rec[10 + a] = kc[5 + a]; rec[13 + a] = ka[5 + a]; }
          }
          ntr += 1;
        }
        continue;
      }

      /* GetRestartCandidate (Section 3.2) */
      double r_cur, r_avg;
      double mu_cur = mu_of(&s, &z, x0r, y0r, omega, &r_cur);
      double mu_avg = mu_of(&s, &zbar, x0r, y0r, omega, &r_avg);
      if (trace_on())
        fprintf(stderr, "  kkt cur %.6e %.6e %.6e avg %.6e %.6e %.6e\n", kc[5], kc[6], kc[7], ka[5], ka[6], ka[7]);
      /* restart_to_current = 0: always the average (Appendix C.2, theory mode) */
      const int to_cur = o->restart_to_current ? mu_cur < mu_avg : 0;
      const iterate *cand = to_cur ? &z : &zbar;
      double muc = to_cur ? mu_cur : mu_avg;
      /* restart criteria (i), (ii), (iii) */
      restart = or_restart_check(muc, mu0, muc_prev, t, k, o->beta_suff, o->beta_nec, o->beta_art) != 0;
      if (trace_on())
        fprintf(stderr, "k=%lld t=%lld mu_cur=%.3e mu_avg=%.3e mu0=%.3e muc_prev=%.3e restart=%d omega=%.4g eta=%.4g\n",
                (long long)k, (long long)t, mu_cur, mu_avg, mu0, muc_prev, restart, omega, eta_hat);
      muc_prev = muc;
      if (trace && ntr < trace_cap) {
        double *rec = trace + (size_t)ntr * OR_TRACE_LEN;
        rec[0] = (double)k;
        rec[1] = (double)t;
        rec[2] = mu_cur;
        rec[3] = mu_avg;
        rec[4] = mu0;
        rec[5] = cand == &z ? 0.0 : 1.0;
        rec[6] = (double)restart;
        rec[7] = omega;
        rec[8] = r_cur;
        rec[9] = r_avg;
        for (int a = 0; a < 3; ++a) { rec[10 + a] = kc[5 + a]; rec[13 + a] = ka[5 + a]; }
      }
      ntr += 1;
      if (!restart) continue;

      /* restart the outer loop at the candidate; Algorithm 3 */
      double dx2 = 0.0, dy2 = 0.0;
      for (int32_t j = 0; j < n; ++j) dx2 += (cand->x[j] - x0r[j]) * (cand->x[j] - x0r[j]);
      for (int32_t i = 0; i < m; ++i) dy2 += (cand->y[i] - y0r[i]) * (cand->y[i] - y0r[i]);
      double Dx = sqrt(dx2), Dy = sqrt(dy2);
      if (cand != &z) copy_iterate(&s, &z, cand);
      if (trace_on()) fprintf(stderr, "  restart to %s: Dx=%.4e Dy=%.4e\n", cand == &z ? "current" : "average", Dx, Dy);
      if (o->pw_update) omega = or_primal_weight(omega, Dx, Dy, o->pw_theta, o->eps_zero);
      if (trace && ntr - 1 < trace_cap) trace[(size_t)(ntr - 1) * OR_TRACE_LEN + 7] = omega;
      /* mu_0 of the new outer loop: mu_n(z^{n,0}, z^{n-1,0}) under the new omega */
      mu0 = mu_of(&s, &z, x0r, y0r, omega, NULL);
      memcpy(x0r, z.x, sizeof(double) * (size_t)n);
      memcpy(y0r, z.y, sizeof(double) * (size_t)m);
      restarts += 1;
    }
  }

  if (status != OR_OPTIMAL) { ret = &z; terminated(lp, &s, &z, o->eps, kkt, xo, yo); }
  else terminated(lp, &s, ret, o->eps, kkt, xo, yo);
  memcpy(x_out, xo, sizeof(double) * (size_t)n);
  memcpy(y_out, yo, sizeof(double) * (size_t)m);
  fill_result(res, kkt);
  res->status = status;
  res->iters = k;
  res->kkt_passes = kkt_passes;
  res->restarts = restarts;
  res->omega = omega;
  res->eta = eta_hat;
  res->returned_average = ret_avg;
  if (trace_n) *trace_n = ntr;

  free_iterate(&z); free_iterate(&zp); free_iterate(&zbar);
  free(sx); free(sy); free(x0r); free(y0r); free(xo); free(yo);
  scaled_free(&s);
}

/* ----------------------------------------------------- Appendix A PDHG */

void or_pdhg_fixed(const or_lp *lp, double eta, double omega, int64_t T, double *x, double *y) {
  int32_t m = lp->m, n = lp->n;
  double *KTy = dalloc((size_t)n), *xn = dalloc((size_t)n), *xe = dalloc((size_t)n),
         *Kxe = dalloc((size_t)m);
  double tau = eta / omega, sigma = eta * omega;
  for (int64_t t = 0; t < T; ++t) {
    spmv_t(m, n, lp->row_ptr, lp->col_idx, lp->val, y, KTy);
    for (int32_t j = 0; j < n; ++j) xn[j] = clip(x[j] - tau * (lp->c[j] - KTy[j]), lp->l[j], lp->u[j]);
    for (int32_t j = 0; j < n; ++j) xe[j] = 2.0 * xn[j] - x[j];
    spmv(m, lp->row_ptr, lp->col_idx, lp->val, xe, Kxe);
    for (int32_t i = 0; i < m; ++i) {
      double v = y[i] + sigma * (lp->q[i] - Kxe[i]);
      double lo = ylo_of(lp, i);
      y[i] = v > lo ? v : lo;
    }
    memcpy(x, xn, sizeof(double) * (size_t)n);
  }
  free(KTy); free(xn); free(xe); free(Kxe);
}

/* ------------------------------------------------------- unrolled PDHG */

static void unroll_start(const scaled_lp *s, const double *x0, const double *y0, double *x, double *y) {
  for (int32_t j = 0; j < s->n; ++j) x[j] = clip(x0 ? x0[j] / s->D2[j] : 0.0, s->l[j], s->u[j]);
  for (int32_t i = 0; i < s->m; ++i) {
    double v = y0 ? y0[i] / s->D1[i] : 0.0;
    y[i] = v > s->ylo[i] ? v : s->ylo[i];
  }
}

void or_unroll_schedule(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                        int64_t T, const double *x0, const double *y0,
                        double *eta_out, double *omega_out, double *x_out, double *y_out) {
  scaled_lp s;
  scaled_build(lp, ruiz_iters, pock_chambolle, &s);
  int32_t m = s.m, n = s.n, nnz = lp->row_ptr[m];
  iterate z, zp;
  alloc_iterate(&s, &z);
  alloc_iterate(&s, &zp);
  unroll_start(&s, x0, y0, z.x, z.y);
  K_mul(&s, z.x, z.Kx);
  KT_mul(&s, z.y, z.KTy);
  double kmax = 0.0;
  for (int32_t k = 0; k < nnz; ++k) kmax = fabs(s.v[k]) > kmax ? fabs(s.v[k]) : kmax;
  double eta_hat = kmax > 0.0 ? 1.0 / kmax : 1.0;
  double omega = init_primal_weight(&s, 1e-10);
  for (int64_t k = 0; k < T; ++k) {
    double eta = eta_hat, eb, en;
    int bad = 0;
    for (int a = 0; a < 64; ++a) {
      pdhg_attempt(&s, &z, &zp, eta, omega, k, &eb, &en, &bad);
      if (bad || eta <= eb) break;
      eta = en;
    }
    eta_out[k] = eta;
    eta_hat = en;
    copy_iterate(&s, &z, &zp);
  }
  *omega_out = omega;
  for (int32_t j = 0; j < n; ++j) x_out[j] = s.D2[j] * z.x[j];
  for (int32_t i = 0; i < m; ++i) y_out[i] = s.D1[i] * z.y[i];
  free_iterate(&z);
  free_iterate(&zp);
  scaled_free(&s);
}

void or_unroll_forward(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                       int64_t T, const double *eta, double omega, const double *x0,
                       const double *y0, double *x_out, double *y_out) {
  scaled_lp s;
  scaled_build(lp, ruiz_iters, pock_chambolle, &s);
  int32_t m = s.m, n = s.n;
  double *x = dalloc((size_t)n), *y = dalloc((size_t)m), *xn = dalloc((size_t)n),
         *KTy = dalloc((size_t)n), *xe = dalloc((size_t)n), *Kxe = dalloc((size_t)m);
  unroll_start(&s, x0, y0, x, y);
  for (int64_t t = 0; t < T; ++t) {
    double tau = eta[t] / omega, sigma = eta[t] * omega;
    KT_mul(&s, y, KTy);
    for (int32_t j = 0; j < n; ++j) xn[j] = clip(x[j] - tau * (s.c[j] - KTy[j]), s.l[j], s.u[j]);
    for (int32_t j = 0; j < n; ++j) xe[j] = 2.0 * xn[j] - x[j];
    K_mul(&s, xe, Kxe);
    for (int32_t i = 0; i < m; ++i) {
      double v = y[i] + sigma * (s.q[i] - Kxe[i]);
      y[i] = v > s.ylo[i] ? v : s.ylo[i];
    }
    memcpy(x, xn, sizeof(double) * (size_t)n);
  }
  for (int32_t j = 0; j < n; ++j) x_out[j] = s.D2[j] * x[j];
  for (int32_t i = 0; i < m; ++i) y_out[i] = s.D1[i] * y[i];
  free(x); free(y); free(xn); free(KTy); free(xe); free(Kxe);
  scaled_free(&s);
}

/* Reverse mode over the stored iterates.  With v_t = x_t - tau (c - K^T y_t),
 * x_{t+1} = clip(v_t), w_t = y_t + sigma (q - K (2 x_{t+1} - x_t)),
 * y_{t+1} = max(w_t, ylo), and adjoints xb (of x_{t+1}), yb (of y_{t+1}):
 *   h   = [w_t > ylo] * yb
 *   xb' = xb - 2 sigma K^T h                 (total adjoint of x_{t+1})
 *   g   = [l < v_t < u] * xb'
 *   dq += sigma h;  dc -= tau g
 *   dK_ij += -sigma h_i (2 x_{t+1} - x_t)_j + tau y_t,i g_j
 *   xb_t = g + sigma K^T h;   yb_t = h + tau K g
 * Gradients with respect to the original data follow from c~ = D2 c,
 * q~ = D1 q, K~_ij = D1_i K_ij D2_j and x = D2 x~, y = D1 y~ (D fixed). */
void or_unroll_vjp(const or_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle,
                   int64_t T, const double *eta, double omega, const double *x0,
                   const double *y0, const double *gx_T, const double *gy_T,
                   double *dc, double *dq, double *dK) {
  scaled_lp s;
  scaled_build(lp, ruiz_iters, pock_chambolle, &s);
  int32_t m = s.m, n = s.n, nnz = lp->row_ptr[m];
  double *X = dalloc((size_t)(T + 1) * (size_t)n), *Y = dalloc((size_t)(T + 1) * (size_t)m);
  double *KTy = dalloc((size_t)n), *xe = dalloc((size_t)n), *Kxe = dalloc((size_t)m);
  unroll_start(&s, x0, y0, X, Y);
  for (int64_t t = 0; t < T; ++t) {
    const double *x = X + t * n, *y = Y + t * m;
    double *xn = X + (t + 1) * n, *yn = Y + (t + 1) * m;
    double tau = eta[t] / omega, sigma = eta[t] * omega;
    KT_mul(&s, y, KTy);
    for (int32_t j = 0; j < n; ++j) xn[j] = clip(x[j] - tau * (s.c[j] - KTy[j]), s.l[j], s.u[j]);
    for (int32_t j = 0; j < n; ++j) xe[j] = 2.0 * xn[j] - x[j];
    K_mul(&s, xe, Kxe);
    for (int32_t i = 0; i < m; ++i) {
      double v = y[i] + sigma * (s.q[i] - Kxe[i]);
      yn[i] = v > s.ylo[i] ? v : s.ylo[i];
    }
  }
  double *xb = dalloc((size_t)n), *yb = dalloc((size_t)m), *h = dalloc((size_t)m),
         *g = dalloc((size_t)n), *KTh = dalloc((size_t)n), *Kg = dalloc((size_t)m);
  double *dcs = dalloc((size_t)n), *dqs = dalloc((size_t)m), *dKs = dalloc((size_t)nnz);
  for (int32_t j = 0; j < n; ++j) xb[j] = s.D2[j] * gx_T[j];
  for (int32_t i = 0; i < m; ++i) yb[i] = gy_T ? s.D1[i] * gy_T[i] : 0.0;
  for (int64_t t = T - 1; t >= 0; --t) {
    const double *x = X + t * n, *y = Y + t * m, *xn = X + (t + 1) * n;
    double tau = eta[t] / omega, sigma = eta[t] * omega;
    /* recompute the pre-projection values of step t */
    KT_mul(&s, y, KTy);
    for (int32_t j = 0; j < n; ++j) xe[j] = 2.0 * xn[j] - x[j];
    K_mul(&s, xe, Kxe);
    for (int32_t i = 0; i < m; ++i) {
      double w = y[i] + sigma * (s.q[i] - Kxe[i]);
      h[i] = (w > s.ylo[i]) ? yb[i] : 0.0;
    }
    KT_mul(&s, h, KTh);
    for (int32_t j = 0; j < n; ++j) {
      double v = x[j] - tau * (s.c[j] - KTy[j]);
      double xbt = xb[j] - 2.0 * sigma * KTh[j];
      g[j] = (v > s.l[j] && v < s.u[j]) ? xbt : 0.0;
    }
    K_mul(&s, g, Kg);
    for (int32_t i = 0; i < m; ++i) dqs[i] += sigma * h[i];
    for (int32_t j = 0; j < n; ++j) dcs[j] -= tau * g[j];
    for (int32_t i = 0; i < m; ++i)
      for (int32_t k = s.rp[i]; k < s.rp[i + 1]; ++k) {
        int32_t j = s.ci[k];
        dKs[k] += -sigma * h[i] * xe[j] + tau * y[i] * g[j];
      }
    for (int32_t j = 0; j < n; ++j) xb[j] = g[j] + sigma * KTh[j];
    for (int32_t i = 0; i < m; ++i) yb[i] = h[i] + tau * Kg[i];
  }
  for (int32_t j = 0; j < n; ++j) dc[j] = s.D2[j] * dcs[j];
  for (int32_t i = 0; i < m; ++i) dq[i] = s.D1[i] * dqs[i];
  for (int32_t i = 0; i < m; ++i)
    for (int32_t k = s.rp[i]; k < s.rp[i + 1]; ++k) dK[k] = s.D1[i] * s.D2[s.ci[k]] * dKs[k];
  free(X); free(Y); free(KTy); free(xe); free(Kxe);
  free(xb); free(yb); free(h); free(g); free(KTh); free(Kg);
  free(dcs); free(dqs); free(dKs);
  scaled_free(&s);
}

/* ------------------------------------------ refinement correction LP */

void or_correction_lp(const or_lp *lp, const double *xh, const double *yh, double dmax,
                      double *cp, double *qp, double *lp_, double *up, double *ylo,
                      double *dP, double *dD) {
  int32_t m = lp->m, n = lp->n;
  double *Kx = dalloc((size_t)m), *KTy = dalloc((size_t)n);
  spmv(m, lp->row_ptr, lp->col_idx, lp->val, xh, Kx);
  spmv_t(m, n, lp->row_ptr, lp->col_idx, lp->val, yh, KTy);
  double pv = 0.0, dv = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    double r = lp->q[i] - Kx[i];
    double viol = lp->ineq[i] ? (r > 0.0 ? r : 0.0) : fabs(r);
    if (viol > pv) pv = viol;
    if (lp->ineq[i]) {
      double lo = ylo_of(lp, i);
      if (lo - yh[i] > dv) dv = lo - yh[i];
    }
  }
  for (int32_t j = 0; j < n; ++j) {
    if (lp->l[j] - xh[j] > pv) pv = lp->l[j] - xh[j];
    if (xh[j] - lp->u[j] > pv) pv = xh[j] - lp->u[j];
    double rc = lp->c[j] - KTy[j];
    int lf = isfinite(lp->l[j]), uf = isfinite(lp->u[j]);
    double lam;
    if (!lf && !uf) lam = 0.0;
    else if (!lf) lam = rc < 0.0 ? rc : 0.0;
    else if (!uf) lam = rc > 0.0 ? rc : 0.0;
    else lam = rc;
    if (fabs(rc - lam) > dv) dv = fabs(rc - lam);
  }
  double P = pv > 1.0 / dmax ? 1.0 / pv : dmax;
  double D = dv > 1.0 / dmax ? 1.0 / dv : dmax;
  if (P < 1.0) P = 1.0;
  if (D < 1.0) D = 1.0;
  for (int32_t j = 0; j < n; ++j) {
    cp[j] = D * (lp->c[j] - KTy[j]);
    lp_[j] = P * (lp->l[j] - xh[j]);
    up[j] = P * (lp->u[j] - xh[j]);
  }
  for (int32_t i = 0; i < m; ++i) {
    qp[i] = P * (lp->q[i] - Kx[i]);
    ylo[i] = lp->ineq[i] ? -D * (yh[i] - ylo_of(lp, i)) : -INFINITY;
  }
  *dP = P;
  *dD = D;
  free(Kx);
  free(KTy);
}
