// The iteration of Algorithm 1 on the device, templated on the arithmetic of
// the sparse products and vectors (T = double or float; scalars are double).
//
// Per step attempt (Algorithm 2) two kernels run:
//   k_primal  x' = proj_X(x - (eta/omega)(c - K^T y))   (K^T y over K^T rows)
//   k_dual    y' = proj_Y(y + eta*omega (q - 2 K x' + K x))  (K x' over K rows)
//             and, in its last CTA, the step-size test of Eq. (4): accept /
//             reject, eta' and the loop condition of the CUDA graph.
// Both also advance the step-weighted sums of Algorithm 1 (into the other
// ping-pong buffer, so a rejected attempt leaves them untouched).
// Every `eval_every` accepted iterations the evaluation kernels compute
// K^T y, K^T y_avg, K x_avg, the termination test of Eq. (15) on the original
// problem for the current and the average iterate, the normalized duality
// gaps of Section 3.2 (radix selection of the trust-region breakpoint), the
// restart decision (criteria (i)-(iii)) and the primal weight of Algorithm 3.
#include <math.h>
#include <stdlib.h>

#include "common.cuh"
#include <algorithm>

#include "evaluate.cuh"
#include "slab.cuh"
#include "solver.cuh"

namespace pdlp {

// ---------------------------------------------------------------- helpers


// Algorithm 2's test and step-size update (step_update), run by one thread
// after the reductions of an attempt, on the scalars in global memory; the
// factors come from the table k_eval_rows fills for the current chunk.
__device__ void accept_step(Scalars *s, double dx2, double dy2, double inter,
                            cudaGraphConditionalHandle h, int has_cond, double *eta_log) {
  StepCtl c;
  load_step(s, c);
  const long long idx = c.k - s->fac_k0;
  double fr, fg;
  if (idx >= 0 && idx < s->eval_every && idx < kMaxEval) {
    fr = s->fac_tab[0][idx];
    fg = s->fac_tab[1][idx];
  } else {
    const double kk = (double)(c.k + 1);
    fr = 1.0 - pow(kk + 1.0, -0.3);
    fg = 1.0 + pow(kk + 1.0, -0.6);
  }
  const long long k_before = c.k;
  const double eta_try = c.eta;
  step_update(c, dx2, dy2, inter, fr, fg);
  store_step(s, c);
  if (eta_log && c.k > k_before) eta_log[k_before] = eta_try;
  bool go = c.status == kRunning && c.chunk_acc < s->eval_every && c.k < s->iter_limit &&
            c.attempts < s->attempt_limit;
  if (go && time_up(s)) go = false;
  if (has_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ------------------------------------------------------------ step kernels

template <typename T>
__global__ void __launch_bounds__(kThreads) k_primal(Mat<T> KT, Problem<T> P, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double red[kThreads];
  const Scalars *sc = S.s;
  const int cur = sc->cur;
  const T tau = (T)sc->tau, et = (T)sc->eta;
  const T *x = S.x[cur];
  T *xn = S.x[cur ^ 1];
  const T *xs = S.xs[cur];
  T *xsn = S.xs[cur ^ 1];
  double acc[1] = {0.0};
  const T *const vec[1] = {S.y[cur]};
  spmv_warp<T, 1>(KT, vec, sm, acc, [&](int j, const T(&g)[1], double(&a)[1]) {
    const T xj = x[j];
    const T xp = clampv<T>(xj - tau * (P.cs[j] - g[0]), P.ls[j], P.us[j]);
    xn[j] = xp;
    xsn[j] = xs[j] + et * xp;
    const T d = xp - xj;
    a[0] += (double)(d * d);
  });
  block_sum_lean<1>(acc, red);
  if (threadIdx.x == 0) S.part_p[blockIdx.x] = acc[0];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dual(Mat<T> K, Mat<T> KT, Problem<T> P, State<T> S,
                                                   cudaGraphConditionalHandle h, int has_cond) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double red[2 * kThreads];
  Scalars *sc = S.s;
  const int cur = sc->cur;
  const T sig = (T)sc->sigma, et = (T)sc->eta;
  const T *y = S.y[cur], *Kx = S.Kx[cur], *ys = S.ys[cur];
  T *yn = S.y[cur ^ 1], *Kxn = S.Kx[cur ^ 1], *ysn = S.ys[cur ^ 1];
  double acc[2] = {0.0, 0.0};
  const T *const vec[1] = {S.x[cur ^ 1]};
  spmv_warp<T, 1>(K, vec, sm, acc, [&](int i, const T(&s)[1], double(&a)[2]) {
    const T kxn = s[0], kx = Kx[i], yi = y[i], lo = P.ylos[i];
    const T v = yi + sig * (P.qs[i] - T(2) * kxn + kx);
    const T yp = v > lo ? v : lo;
    yn[i] = yp;
    Kxn[i] = kxn;
    ysn[i] = ys[i] + et * yp;
    const T dy = yp - yi, dk = kxn - kx;
    a[0] += (double)(dy * dy);
    a[1] += (double)dy * (double)dk;
  });
  block_sum_lean<2>(acc, red);
  if (threadIdx.x == 0) {
    S.part_d[2 * blockIdx.x] = acc[0];
    S.part_d[2 * blockIdx.x + 1] = acc[1];
  }
  if (last_block(S.tickets + kTicketDual)) {
    double p[1], d[2], lp[1], ld[2];
    sum_partials<1>(S.part_p, KT.nblocks, 1, p, red);
    __syncthreads();
    sum_partials<2>(S.part_d, gridDim.x, 2, d, red);
    __syncthreads();
    sum_long_rows<1>(KT, lp, red);
    __syncthreads();
    sum_long_rows<2>(K, ld, red);
    if (threadIdx.x == 0) accept_step(sc, p[0] + lp[0], d[0] + ld[0], d[1] + ld[1], h, has_cond, S.eta_log);
  }
}

// Slab step kernels (slab.cuh): the same half-steps and epilogues as
// k_primal / k_dual over fixed-size slabs, one warp per slab; the dual
// kernel's last CTA runs the step test on the partials of both launches
// and the split-row slots, in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kSlabThreads, 5) k_primal_slab(Mat<T> KT, Problem<T> P, State<T> S) {
  __shared__ unsigned bits[kSlabWarps][8];
  __shared__ __align__(16) T srow[kSlabWarps][kSlabNnz];
  __shared__ double red[kSlabThreads];
  const Scalars *sc = S.s;
  const int cur = sc->cur, wid = threadIdx.x >> 5;
  const T tau = (T)sc->tau, et = (T)sc->eta;
  const T *x = S.x[cur];
  T *xn = S.x[cur ^ 1];
  const T *xs = S.xs[cur];
  T *xsn = S.xs[cur ^ 1];
  double acc[1] = {0.0};
  auto epi = [&](int j, T g, double(&a)[1]) {
    const T xj = x[j];
    const T xp = clampv<T>(xj - tau * (P.cs[j] - g), P.ls[j], P.us[j]);
    xn[j] = xp;
    xsn[j] = xs[j] + et * xp;
    const T d = xp - xj;
    a[0] += (double)(d * d);
  };
  for (int s = slab_begin(KT.nslab) + wid, se = slab_begin(KT.nslab, 1); s < se; s += kSlabWarps)
    slab_warp<T, 1>(KT, s, S.y[cur], bits[wid], srow[wid], acc, epi);
  block_sum_lean<1>(acc, red);
  if (threadIdx.x == 0) S.part_sp[blockIdx.x] = acc[0];
  if (KT.ndefer > 0 && last_block(S.tickets + kTicketSlabPrimal)) finish_deferred<T, 1>(KT, epi, red);
}

template <typename T>
__global__ void __launch_bounds__(kSlabThreads, 5) k_dual_slab(Mat<T> K, Mat<T> KT, Problem<T> P, State<T> S,
                                                            cudaGraphConditionalHandle h, int has_cond) {
  __shared__ unsigned bits[kSlabWarps][8];
  __shared__ __align__(16) T srow[kSlabWarps][kSlabNnz];
  __shared__ double red[2 * kSlabThreads];
  Scalars *sc = S.s;
  const int cur = sc->cur, wid = threadIdx.x >> 5;
  const T sig = (T)sc->sigma, et = (T)sc->eta;
  const T *y = S.y[cur], *Kx = S.Kx[cur], *ys = S.ys[cur];
  T *yn = S.y[cur ^ 1], *Kxn = S.Kx[cur ^ 1], *ysn = S.ys[cur ^ 1];
  double acc[2] = {0.0, 0.0};
  auto epi = [&](int i, T kxn, double(&a)[2]) {
    const T kx = Kx[i], yi = y[i], lo = P.ylos[i];
    const T v = yi + sig * (P.qs[i] - T(2) * kxn + kx);
    const T yp = v > lo ? v : lo;
    yn[i] = yp;
    Kxn[i] = kxn;
    ysn[i] = ys[i] + et * yp;
    const T dy = yp - yi, dk = kxn - kx;
    a[0] += (double)(dy * dy);
    a[1] += (double)dy * (double)dk;
  };
  for (int s = slab_begin(K.nslab) + wid, se = slab_begin(K.nslab, 1); s < se; s += kSlabWarps)
    slab_warp<T, 2>(K, s, S.x[cur ^ 1], bits[wid], srow[wid], acc, epi);
  block_sum_lean<2>(acc, red);
  if (threadIdx.x == 0) {
    S.part_sd[2 * blockIdx.x] = acc[0];
    S.part_sd[2 * blockIdx.x + 1] = acc[1];
  }
  if (last_block(S.tickets + kTicketDual)) {
    if (K.ndefer > 0) finish_deferred<T, 2>(K, epi, red);
    double p[1], d[2], lp[1], ld[2];
    sum_partials<1>(S.part_sp, KT.slab_grid, 1, p, red);
    __syncthreads();
    sum_partials<2>(S.part_sd, gridDim.x, 2, d, red);
    __syncthreads();
    sum_split_rows<1>(KT, lp, red);
    __syncthreads();
    sum_split_rows<2>(K, ld, red);
    if (threadIdx.x == 0) accept_step(sc, p[0] + lp[0], d[0] + ld[0], d[1] + ld[1], h, has_cond, S.eta_log);
  }
}

// CTAs of the slab launches of a precision: the number of CTAs resident at
// once (SMs x occupancy), or fewer when there are fewer slab groups; each CTA
// takes a contiguous range of slabs (slab_begin), its warps interleaved.
template <typename T>
cudaError_t plan_slab_grid(Mat<T> &K, Mat<T> &KT) {
  int dev = 0, sms = 0, occ_p = 0, occ_d = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, k_primal_slab<T>, kSlabThreads, 0))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, k_dual_slab<T>, kSlabThreads, 0))) return e;
  const int resident = sms * std::max(1, std::min(occ_p, occ_d));
  KT.slab_grid = std::max(1, std::min(slab_ctas(KT.nslab), resident));
  K.slab_grid = std::max(1, std::min(slab_ctas(K.nslab), resident));
  return cudaSuccess;
}
template cudaError_t plan_slab_grid<double>(Mat<double> &, Mat<double> &);
template cudaError_t plan_slab_grid<float>(Mat<float> &, Mat<float> &);

// One step attempt on the engine the matrices select (slab kernels or the
// warp-chunk kernels), as graph nodes when has_cond.
template <typename T>
void launch_attempt(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                    cudaGraphConditionalHandle h, int has_cond, cudaStream_t st) {
  if (K.slab_on) {
    k_primal_slab<T><<<KT.slab_grid, kSlabThreads, 0, st>>>(KT, P, S);
    k_dual_slab<T><<<K.slab_grid, kSlabThreads, 0, st>>>(K, KT, P, S, h, has_cond);
    return;
  }
  if (KT.nblocks > 0) k_primal<T><<<KT.nblocks, kThreads, spmv_smem_bytes<T>(1), st>>>(KT, P, S);
  k_dual<T><<<K.nblocks, kThreads, spmv_smem_bytes<T>(1), st>>>(K, KT, P, S, h, has_cond);
}

// -------------------------------------- Malitsky-Pock line search (App. C.1)
//
// One trial per pass of the inner loop: k_mp_primal (K^T y, x' =
// proj_X(x - (eta_k / omega)(c - K^T y))) and k_mp_kx (K x') run in the
// first trial of an iteration only; k_mp_dual forms y_hat from the stored
// K x' with the trial's eta_hat, theta_hat; k_mp_cols takes K^T y_hat and
// ||K^T (y_hat - y)||^2 (and the average sums of the columns); k_mp_test
// accepts or shrinks eta_hat.  The buffers of index cur ^ 1 hold the trial.

template <typename T>
__global__ void __launch_bounds__(kThreads) k_mp_primal(Mat<T> KT, Problem<T> P, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  const Scalars *sc = S.s;
  if (sc->mp_trial) return;  // uniform over the grid
  const int cur = sc->cur;
  const T tau = (T)(sc->mp_eta_k / sc->omega);
  const T *x = S.x[cur];
  T *xn = S.x[cur ^ 1], *kty = S.KTy_cur;
  double acc[1] = {0.0};
  const T *const vec[1] = {S.y[cur]};
  spmv_warp<T, 1>(KT, vec, sm, acc, [&](int j, const T(&g)[1], double(&)[1]) {
    kty[j] = g[0];
    xn[j] = clampv<T>(x[j] - tau * (P.cs[j] - g[0]), P.ls[j], P.us[j]);
  });
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_mp_kx(Mat<T> K, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  const Scalars *sc = S.s;
  if (sc->mp_trial) return;
  const int cur = sc->cur;
  T *kxn = S.Kx[cur ^ 1];
  double acc[1] = {0.0};
  const T *const vec[1] = {S.x[cur ^ 1]};
  spmv_warp<T, 1>(K, vec, sm, acc, [&](int i, const T(&v)[1], double(&)[1]) { kxn[i] = v[0]; });
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_mp_dual(Problem<T> P, State<T> S) {
  __shared__ double red[kThreads / 32];
  const Scalars *sc = S.s;
  const int cur = sc->cur;
  const double eh = sc->mp_eh, th = sc->mp_th;
  const T sg = (T)(sc->omega * eh), tht = (T)th, et = (T)eh;
  const T *y = S.y[cur], *kx = S.Kx[cur], *kxn = S.Kx[cur ^ 1], *ys = S.ys[cur];
  T *yn = S.y[cur ^ 1], *ysn = S.ys[cur ^ 1];
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.m; i += gridDim.x * blockDim.x) {
    const T kb = kxn[i] + tht * (kxn[i] - kx[i]);  // K (x' + theta_hat (x' - x))
    const T v = y[i] + sg * (P.qs[i] - kb), lo = P.ylos[i];
    const T yp = v > lo ? v : lo;
    yn[i] = yp;
    ysn[i] = ys[i] + et * yp;
    const double d = (double)yp - (double)y[i];
    acc[0] += d * d;
  }
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) S.part_d[blockIdx.x] = acc[0];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_mp_cols(Mat<T> KT, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double red[kThreads / 32];
  const Scalars *sc = S.s;
  const int cur = sc->cur;
  const T et = (T)sc->mp_eh;
  const T *kty = S.KTy_cur, *xn = S.x[cur ^ 1], *xs = S.xs[cur];
  T *xsn = S.xs[cur ^ 1];
  double acc[1] = {0.0};
  const T *const vec[1] = {S.y[cur ^ 1]};
  spmv_warp<T, 1>(KT, vec, sm, acc, [&](int j, const T(&g)[1], double(&a)[1]) {
    const double d = (double)g[0] - (double)kty[j];
    a[0] += d * d;
    xsn[j] = xs[j] + et * xn[j];
  });
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) S.part_p[blockIdx.x] = acc[0];
}

// The line-search test of one trial (one CTA): sums the partials in a fixed
// order, then thread 0 accepts (eta_{k+1} = eta_hat, theta_{k+1} = theta_hat,
// next candidate from the interpolation coefficient) or shrinks eta_hat.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mp_test(Mat<T> KT, State<T> S, int nparts_p, int nparts_d,
                                                      cudaGraphConditionalHandle h, int has_cond) {
  __shared__ double red[kThreads / 32];
  Scalars *s = S.s;
  double dk[1], dy[1], lk[1];
  sum_partials<1>(S.part_p, nparts_p, 1, dk, red);
  __syncthreads();
  sum_long_rows<1>(KT, lk, red);
  __syncthreads();
  sum_partials<1>(S.part_d, nparts_d, 1, dy, red);
  if (threadIdx.x != 0) return;
  const double dk2 = dk[0] + lk[0], dy2 = dy[0];
  const double eh = s->mp_eh;
  s->attempts += 1;
  s->dx2 = dk2;
  s->dy2 = dy2;
  if (!isfinite(dk2) || !isfinite(dy2) || !isfinite(eh)) {
    s->status = kNumErr;
  } else if (eh * sqrt(dk2) <= s->mp_bf * sqrt(dy2)) {
    s->cur ^= 1;
    s->sum_eta += eh;
    s->k += 1;
    s->t += 1;
    s->chunk_acc += 1;
    s->mp_eta_k = eh;
    s->mp_theta = s->mp_th;
    s->mp_trial = 0;
    s->mp_eh = s->mp_eta_k + s->mp_ic * (sqrt(1.0 + s->mp_theta) - 1.0) * s->mp_eta_k;
    s->mp_th = s->mp_eta_k / s->mp_eh;
  } else {
    s->mp_trial += 1;
    s->mp_eh = s->mp_eh * s->mp_df;
    s->mp_th = s->mp_eta_k / s->mp_eh;
  }
  s->eta = s->mp_eta_k;
  s->tau = s->eta * s->inv_omega;
  s->sigma = s->eta * s->omega;
  bool go = s->status == kRunning && s->chunk_acc < s->eval_every && s->k < s->iter_limit &&
            s->attempts < s->attempt_limit;
  if (go && time_up(s)) go = false;
  if (has_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ------------------------------------------------------ evaluation kernels

// Columns: K^T y (current) and K^T ys (sum for the average) in one pass, and
// the column terms of Eq. (15) for both candidates.
// Partial layout per CTA (8): [cand][pobj, dres^2, dobj(lambda), |x - x0|^2].

// The per-CTA partials of an evaluation (8 terms per CTA of k_eval_cols and
// of k_eval_rows) are summed in a fixed-order two-level tree: the last CTA of
// each group of kEvalGroup CTAs sums its group's partials (one warp per
// term) into the group's first slot, and the last group to finish, over both
// kernels (which may run concurrently), sums the group partials and the
// long-row slots and finishes the evaluation.  A one-CTA sum of all partials
// would cost thousands of float64 instructions on one SM.
constexpr int kEvalGroup = 32;
static_assert(kThreads == 8 * 32, "one warp per evaluation term");

template <typename T>
__device__ __forceinline__ unsigned eval_groups(const Mat<T> &K, const Mat<T> &KT) {
  const int gc = KT.nblocks > 0 ? (KT.nblocks + kEvalGroup - 1) / kEvalGroup : 0;
  return (unsigned)(gc + (K.nblocks + kEvalGroup - 1) / kEvalGroup);
}

// Sums of two terms (t0, t0 + 1) over `ng` group partials (stride kEvalGroup
// CTAs) and the long rows of A, by one warp, valid in lane 0: every load is
// issued before any sum (one round trip), and each term takes one shuffle
// reduction.
template <typename T>
__device__ __forceinline__ void eval_terms2(const double *part, int ng, const Mat<T> &A, int t0, double (&out)[2]) {
  const int lane = threadIdx.x & 31;
  double acc[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[q][u] = 0.0;
  for (int g0 = lane; g0 < ng; g0 += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int g = g0 + 32 * u;
      if (g < ng) {
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q][u] += __ldcg(part + (size_t)g * kEvalGroup * 8 + t0 + q);
      }
    }
  }
  for (int r0 = lane; r0 < A.nlong; r0 += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 32 * u;
      if (r < A.nlong) {
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q][u] += __ldcg(A.lr_acc + (size_t)r * kLrAcc + t0 + q);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    double t = (acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    out[q] = t;
  }
}

// Called by every CTA of k_eval_cols (cols = true) and k_eval_rows after its
// partials are stored at part[8 blockIdx.x].
template <typename T>
__device__ void eval_arrive(const Mat<T> &K, const Mat<T> &KT, const State<T> &S, bool cols) {
  __shared__ double ecr[16];
  double *part = cols ? S.part_ec : S.part_er;
  const int nb = cols ? KT.nblocks : K.nblocks;
  const int grp = blockIdx.x / kEvalGroup, g0 = grp * kEvalGroup;
  const int gsize = nb - g0 < kEvalGroup ? nb - g0 : kEvalGroup;
  const int gc = KT.nblocks > 0 ? (KT.nblocks + kEvalGroup - 1) / kEvalGroup : 0;
  if (!last_of(S.gtickets + (cols ? grp : gc + grp), (unsigned)gsize)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp = term
  double v = lane < gsize ? __ldcg(part + (size_t)(g0 + lane) * 8 + warp) : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // every term of the group is read before its first slot is overwritten
  if (lane == 0) part[(size_t)g0 * 8 + warp] = v;
  if (!last_of(S.tickets + kTicketEvalRows, eval_groups(K, KT))) return;
  // warp w: terms 2w and 2w + 1 of [column terms (8), row terms (8)]
  double t2[2];
  if (warp < 4) eval_terms2(S.part_ec, gc, KT, 2 * warp, t2);
  else eval_terms2(S.part_er, (K.nblocks + kEvalGroup - 1) / kEvalGroup, K, 2 * warp - 8, t2);
  if (lane == 0) {
    ecr[2 * warp] = t2[0];
    ecr[2 * warp + 1] = t2[1];
  }
  __syncthreads();
  eval_finish(S.s, ecr, S.trace);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_eval_cols(Mat<T> K, Mat<T> KT, Problem<T> P, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  const Scalars *sc = S.s;
  const int cur = sc->cur;
  const bool avg = sc->sum_eta > 0.0;
  const double inv = avg ? 1.0 / sc->sum_eta : 0.0;
  const T *x = S.x[cur], *xs = S.xs[cur], *x0 = S.x0;
  double acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = 0.0;
  const T *const vec[2] = {S.y[cur], S.ys[cur]};
  spmv_warp<T, 2>(KT, vec, sm, acc, [&](int j, const T(&g)[2], double(&acc)[8]) {
    S.KTy_cur[j] = g[0];
    S.KTys[j] = g[1];
    const double D2 = P.D2[j], iD2 = P.D2inv[j], cj = P.c[j], lj = P.l[j], uj = P.u[j], xr = (double)x0[j];
    // Lambda_j from the finiteness of l_j and u_j (Section 2); lambda =
    // proj_Lambda(rc) is rc or 0, so rc - lambda is 0 (rc - rc) or rc, and
    // at most one of l_j lambda+ and u_j lambda- is nonzero: the same values
    // as the plain formulas, with bit tests instead of float64 compares
    const bool lf = !d_is_neginf(lj), uf = !d_is_posinf(uj);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 1 && !avg) break;
      const double xt = c == 0 ? (double)x[j] : (double)xs[j] * inv;
      const double kt = c == 0 ? (double)g[0] : (double)g[1] * inv;
      const double xo = D2 * xt, rc = cj - kt * iD2;
      const bool lam_rc = lf ? (uf || d_gt0(rc)) : (uf && d_lt0(rc));
      const double lam = lam_rc ? rc : 0.0;
      const double d = lam_rc ? (d_finite(rc) ? 0.0 : __longlong_as_double(0x7ff8000000000000ll)) : rc;
      acc[4 * c + 0] += cj * xo;
      acc[4 * c + 1] = fma(d, d, acc[4 * c + 1]);
      if (d_gt0(lam) || d_lt0(lam)) acc[4 * c + 2] = __dadd_rn(acc[4 * c + 2], __dmul_rn(d_gt0(lam) ? lj : uj, lam));
      acc[4 * c + 3] += (xt - xr) * (xt - xr);
    }
  });
  // the staging area is free now: few float64 adds (float64 is slow on this part)
  block_sum_lean<8>(acc, reinterpret_cast<double *>(sm));
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) S.part_ec[8 * blockIdx.x + a] = acc[a];
  }
  eval_arrive(K, KT, S, true);
}


// Rows: K xs (for K x_avg) and the row terms of Eq. (15) for both candidates.
// Partial layout per CTA (8): [cand][pres^2, dobj(q^T y), |y - y0|^2, pobj extra].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_eval_rows(Mat<T> K, Mat<T> KT, Problem<T> P, State<T> S) {
  extern __shared__ __align__(16) char sm[];
  Scalars *sc = S.s;
  const int cur = sc->cur;
  const bool avg = sc->sum_eta > 0.0;
  const double inv = avg ? 1.0 / sc->sum_eta : 0.0;
  const T *y = S.y[cur], *ys = S.ys[cur], *Kx = S.Kx[cur], *y0 = S.y0;
  if (blockIdx.x == 0) {
    // Algorithm 2's factors for the next chunk's steps (k does not change
    // until then), computed here, where their float64 pow overlaps the
    // products, rather than in the one-CTA k_finish
    const long long k0 = sc->k;
    const int ne = sc->eval_every < kMaxEval ? sc->eval_every : kMaxEval;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
      const double kk = (double)(k0 + i + 1);
      sc->fac_tab[0][i] = 1.0 - pow(kk + 1.0, -0.3);
      sc->fac_tab[1][i] = 1.0 + pow(kk + 1.0, -0.6);
    }
    if (threadIdx.x == 0) sc->fac_k0 = k0;
  }
  double acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = 0.0;
  const T *const vec[1] = {S.xs[cur]};
  spmv_warp<T, 1>(K, vec, sm, acc, [&](int i, const T(&s)[1], double(&acc)[8]) {
    S.Kxbar[i] = s[0];
    const double D1 = P.D1[i], iD1 = P.D1inv[i], qi = P.q[i], lo = P.ylo[i], yr = (double)y0[i];
    const bool ineq = !d_is_neginf(lo), lo_nz = d_gt0(lo) || d_lt0(lo);  // bit tests, as in the columns
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 1 && !avg) break;
      const double yt = c == 0 ? (double)y[i] : (double)ys[i] * inv;
      const double kx = c == 0 ? (double)Kx[i] : (double)s[0] * inv;
      double r = qi - kx * iD1;
      if (ineq) {                                 // inequality row
        if (lo_nz) acc[4 * c + 3] += lo * r;      // general dual bound only
        r = d_gt0(r) ? r : 0.0;
      }
      acc[4 * c + 0] += r * r;
      acc[4 * c + 1] += qi * (D1 * yt);
      acc[4 * c + 2] += (yt - yr) * (yt - yr);
    }
  });
  // the staging area is free now: few float64 adds (float64 is slow on this part)
  block_sum_lean<8>(acc, reinterpret_cast<double *>(sm));
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) S.part_er[8 * blockIdx.x + a] = acc[a];
  }
  eval_arrive(K, KT, S, false);
}

// --------------------------------------------- normalized gap (Section 3.2)
//
// For slot s with point z, gradient g = (K^T y - c, q - K x), weight omega and
// radius r, the maximiser of g^T d over ||d||_omega <= r, z + d in Z is
// d(t) = (clip(t g_x/omega, l - x, u - x), clip(t omega g_y, ylo - y, inf)) at
// the t with phi(t) = ||d(t)||^2_omega = r^2.  Item i (a coordinate with
// g_i != 0) stays unclipped until its breakpoint t_i; with a_i (unclipped t^2
// and t coefficient), w_i (clipped contribution to phi) and v_i (clipped
// contribution to g^T d):
//     phi(t) = sum_{t_i <= t} w_i + t^2 sum_{t_i > t} a_i.
// Items with t_i = 0 are clipped for every t > 0 and contribute nothing, so
// they are dropped; items with t_i = +inf (no bound in the direction of g)
// only ever contribute a_i.  The breakpoint is found by a three-pass radix
// selection on the float32 bits of t_i (11, 11, 10 bits): each pass
// histograms (w, v, a) over the digit of the items still in the selected
// bucket, and the last CTA picks the last bucket whose lower edge has
// phi < r^2 (parallel scans in fixed order).

constexpr unsigned kKeyNone = 0xffffffffu;  // no item (g = 0 or t = 0)
constexpr unsigned kKeyInf = 0x7f800000u;   // t = +inf

struct GapItem {
  unsigned key;
  double a, w, v;
};

template <typename T>
__device__ __forceinline__ GapItem gap_item(const Problem<T> &P, const State<T> &S, const Scalars *sc, int slot,
                                            int i, double om, double inv_om) {
  const int cur = sc->cur, n = P.n;
  const double inv = sc->inv_avg;
  GapItem it;
  it.key = kKeyNone;
  it.a = it.w = it.v = 0.0;
  if (i < n) {
    double x, kt;
    if (slot == 0) { x = (double)S.x[cur][i]; kt = (double)S.KTy_cur[i]; }
    else if (slot == 1) { x = (double)S.xs[cur][i] * inv; kt = (double)S.KTys[i] * inv; }
    else { x = (double)S.x[cur][i]; kt = sc->cand == 0 ? (double)S.KTy_cur[i] : (double)S.KTys[i] * inv; }
    const double g = kt - (double)P.cs[i];
    if (g == 0.0) return it;
    // distances to the bounds are >= 0 for a point of Z; the average can sit
    // an ulp outside its box after rounding, which counts as on the bound
    const double dist = g > 0.0 ? (double)P.us[i] - x : x - (double)P.ls[i];
    if (!(dist > 0.0)) return it;
    const double ag = fabs(g);
    it.a = g * g * inv_om;
    if (isinf(dist)) { it.key = kKeyInf; return it; }
    const float tf = (float)(om * dist) / (float)ag;
    if (!(tf > 0.0f)) { it.key = kKeyNone; return it; }
    it.key = __float_as_uint(tf);
    it.w = om * dist * dist;
    it.v = ag * dist;
  } else {
    const int r = i - n;
    double y, kx;
    if (slot == 0) { y = (double)S.y[cur][r]; kx = (double)S.Kx[cur][r]; }
    else if (slot == 1) { y = (double)S.ys[cur][r] * inv; kx = (double)S.Kxbar[r] * inv; }
    else { y = (double)S.y[cur][r]; kx = (double)S.Kx[cur][r]; }
    const double g = (double)P.qs[r] - kx;
    if (g == 0.0) return it;
    const double dist = g > 0.0 ? INFINITY : y - (double)P.ylos[r];
    if (!(dist > 0.0)) return it;
    const double ag = fabs(g);
    it.a = om * g * g;
    if (isinf(dist)) { it.key = kKeyInf; return it; }
    const float tf = (float)dist / ((float)om * (float)ag);
    if (!(tf > 0.0f)) { it.key = kKeyNone; return it; }
    it.key = __float_as_uint(tf);
    it.w = dist * dist * inv_om;
    it.v = ag * dist;
  }
  return it;
}

__device__ __forceinline__ void gap_digits(int pass, int &shift, int &nb, int &pshift) {
  shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
  nb = pass == 2 ? 1024 : 2048;
  pshift = pass == 0 ? 32 : (pass == 1 ? 21 : 10);
}

// The last CTA of a gap pass selects up to two slots at once, one per group
// of kSelThreads threads with its own named barrier.  A float64 instruction
// holds its sub-partition's float64 unit for tens of cycles on this part
// however few lanes are active, so the selection is written for few float64
// instructions per warp: the groups take alternate warps (warp parity), so
// that the two selections run on different sub-partitions; entries are
// spread over as many warps as they fill; prefixes inside a thread are
// sequential; sign, NaN and ordering tests on nonnegative values are integer
// tests on their bits.
constexpr int kSelThreads = 256;
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kSelPer = kGapBuckets / kSelThreads;  // up to 8 buckets, then entries, per thread
constexpr int kSelSmem = 3 * kGapBuckets + kGapBuckets / 2;  // doubles per group (w, v, a, bucket ids)
static_assert(kGapThreads == 2 * kSelThreads, "two selection groups per CTA");
static_assert(1024 % kGapThreads == 0 && kGapBuckets % kGapThreads == 0, "flush ballots: whole warps per bucket");

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kSelThreads) : "memory");
}

// For nonnegative doubles (and +inf) the bit patterns order as the values;
// a NaN pattern orders above +inf.
__device__ __forceinline__ bool nonneg_less(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool nonneg_positive(double a) { return __double_as_longlong(a) > 0ll; }

// Exclusive scans over the first `nwa` warps of group g (group-local warp
// index wg): wex and vex sum tw and tv over lower threads, asuf sums ta over
// higher threads (inclusive scans by shuffles, then the neighbour's inclusive
// value, so no subtraction).  Warps at and above nwa hold no entries and run
// no float64 instruction; every thread of the group must call it.  `sh`
// holds 6 x 32 doubles.
__device__ __forceinline__ void scan3_active(double tw, double tv, double ta, int nwa, int g, int wg, double &wex,
                                             double &vex, double &asuf, double *sh) {
  const int lane = threadIdx.x & 31;
  double xw = tw, xv = tv, xa = ta;
  if (wg < nwa) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double pw = __shfl_up_sync(0xffffffffu, xw, o);
      const double pv = __shfl_up_sync(0xffffffffu, xv, o);
      const double pa = __shfl_down_sync(0xffffffffu, xa, o);
      if (lane >= o) { xw += pw; xv += pv; }
      if (lane + o < 32) xa += pa;
    }
    if (lane == 31) { sh[wg] = xw; sh[32 + wg] = xv; }
    if (lane == 0) sh[64 + wg] = xa;
  }
  if (nwa > 1) {
    group_sync(g);
    if (wg == 0) {  // scans of the warp totals (at most kSelWarps of them)
      double w = lane < nwa ? sh[lane] : 0.0, v = lane < nwa ? sh[32 + lane] : 0.0;
      double a = lane < nwa ? sh[64 + lane] : 0.0;
      for (int o = 1; o < nwa; o <<= 1) {
        const double pw = __shfl_up_sync(0xffffffffu, w, o);
        const double pv = __shfl_up_sync(0xffffffffu, v, o);
        const double pa = __shfl_down_sync(0xffffffffu, a, o);
        if (lane >= o) { w += pw; v += pv; }
        if (lane + o < nwa) a += pa;
      }
      sh[96 + lane] = w;  // inclusive, in the scan direction
      sh[128 + lane] = v;
      sh[160 + lane] = a;
    }
    group_sync(g);
  }
  wex = vex = asuf = 0.0;
  if (wg < nwa) {
    double ew = __shfl_up_sync(0xffffffffu, xw, 1), ev = __shfl_up_sync(0xffffffffu, xv, 1);
    double ea = __shfl_down_sync(0xffffffffu, xa, 1);
    if (lane == 0) ew = ev = 0.0;
    if (lane == 31) ea = 0.0;
    wex = wg > 0 ? sh[96 + wg - 1] + ew : ew;
    vex = wg > 0 ? sh[128 + wg - 1] + ev : ev;
    asuf = wg + 1 < nwa ? sh[160 + wg + 1] + ea : ea;
  }
}

// True when a bucket's three sums are all +0 (bit test: no float64 compare).
__device__ __forceinline__ bool bucket_empty(double w, double v, double a) {
  return (__double_as_longlong(w) | __double_as_longlong(v) | __double_as_longlong(a)) == 0ll;
}

// The slot's value mu = g^T d / r from the clipped sums (Wf, Vf) and the
// unclipped coefficient Aa at the crossing t* (phi(t*) = r^2); r = sqrt(r^2)
// computed beforehand.
__device__ __forceinline__ void gap_final(Scalars *s, int slot, double Wf, double Vf, double Aa, double r2,
                                          double r) {
  double val = Vf;
  if (nonneg_positive(Aa)) {
    const double rem = r2 - Wf;
    val = Vf + sqrt((nonneg_positive(rem) ? rem : 0.0) / Aa) * Aa;
  }
  s->gval[slot] = val;
  s->mu[slot] = val / r;
  s->g_active[slot] = 0;  // finished: later passes skip the slot
}

// Selection over one slot's global histogram ([3][kGapBuckets]: w, v, a) by
// group g of the last CTA, which also clears the histogram for the next
// pass; gin holds the slot's (W, V, A, r^2) below / after the range and
// gpref its key prefix, as they stood when the pass started.  phi at bucket
// lower edges is nondecreasing, and the crossing's clipped set only changes
// at nonempty buckets, so the last NONEMPTY bucket whose lower edge has
// phi < r^2 gives the same partition of the items as the last bucket of any
// kind: the nonempty buckets are compacted in bucket order (ballots and
// integer prefixes) and only they enter the float64 scans.  When the chosen
// bucket holds no item (the crossing falls between nonempty buckets) or this
// is the last digit, the slot's value is final.  `sh` is the group's part of
// the kernel's histogram area (free after the flush), kSelSmem doubles; mk
// the slot's bitmap of nonempty buckets.
__device__ void gap_select(Scalars *s, int slot, int pass, double *gh, unsigned *mk, double *sh, const double *gin,
                           unsigned gpref, int g) {
  int shift, nb, pshift;
  gap_digits(pass, shift, nb, pshift);
  __shared__ double scan_sh[2][6 * 32];
  __shared__ double s_r[2];
  __shared__ unsigned s_word[2][kGapBuckets / 32];
  __shared__ int s_off[2][kGapBuckets / 32 + 1];
  __shared__ int s_ff[2][kSelWarps];
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 6, t = wg * 32 + lane;  // group warps: parity g
  double *cw = sh, *cv = sh + kGapBuckets, *ca = sh + 2 * kGapBuckets;
  int *cb = reinterpret_cast<int *>(sh + 3 * kGapBuckets);
  const double W0 = gin[0], V0 = gin[1], A0 = gin[2], r2 = gin[3];
  // 1. the nonempty buckets, from the slot's bitmap (every CTA's flush sets
  // the bits of the buckets it added to), compacted in bucket order; only
  // they are loaded from the histogram, then cleared with their bits
  constexpr int kWords = kGapBuckets / 32;
  if (t < kWords) {
    const unsigned wv = t < nb / 32 ? __ldcg(mk + t) : 0u;
    s_word[g][t] = wv;
    if (wv) mk[t] = 0u;
  }
  if (wg == kSelWarps - 1 && lane == 0) s_r[g] = sqrt(r2);  // for the final value, off the critical path
  group_sync(g);
  if (wg == 0) {  // exclusive prefix of the 64 word populations
    const int c0 = __popc(s_word[g][2 * lane]), c1 = __popc(s_word[g][2 * lane + 1]);
    int incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int p = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += p;
    }
    const int ex = incl - c0 - c1;
    s_off[g][2 * lane] = ex;
    s_off[g][2 * lane + 1] = ex + c0;
    if (lane == 31) s_off[g][kWords] = incl;
  }
  group_sync(g);
  const int M = s_off[g][kWords];
  {
    const int w = t >> 2, qd = t & 3;  // word w, bits [8 qd, 8 qd + 8)
    const unsigned word = s_word[g][w];
    const unsigned bits = (word >> (8 * qd)) & 0xffu;
    const int ew = s_off[g][w] + __popc(word & ((1u << (8 * qd)) - 1u));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!(bits & (1u << j))) continue;
      const int b = 32 * w + 8 * qd + j;
      const int e = ew + __popc(bits & ((1u << j) - 1u));
      cw[e] = __ldcg(gh + b);
      cv[e] = __ldcg(gh + kGapBuckets + b);
      ca[e] = __ldcg(gh + 2 * kGapBuckets + b);
      cb[e] = b;
      gh[b] = 0.0;
      gh[kGapBuckets + b] = 0.0;
      gh[2 * kGapBuckets + b] = 0.0;
    }
    // zeros after the last entry, up to the end of the last thread's entries
    const int Mp = (M + 32 * kSelPer - 1) / (32 * kSelPer) * (32 * kSelPer);
    for (int e = M + t; e < Mp && e < kGapBuckets; e += kSelThreads) {
      cw[e] = 0.0;
      cv[e] = 0.0;
      ca[e] = 0.0;
      cb[e] = 0;
    }
  }
  group_sync(g);
  if (M == 0) {
    // no item in this digit's range: every edge gives the same partition
    if (t == 0) gap_final(s, slot, W0, V0, A0, r2, s_r[g]);
    return;
  }
  // 2. float64 scans over the M compacted entries: E consecutive ones per
  // thread, E the smallest power of two with M <= E kSelThreads
  // (each warp pays a fixed shuffle scan: as few warps as the entries
  // allow, but not fewer than the group's two sub-partitions can run)
  const int E = M <= 64 ? 1 : (M <= 128 ? 2 : (M <= 256 ? 4 : 8));
  const int nwa = (M + 32 * E - 1) / (32 * E);  // warps holding entries
  const int e0 = t * E;
  const unsigned base = pass == 0 ? 0u : (gpref >> pshift) << pshift;
  // entries past M read as zeros (the compacted area is zero-padded below)
  double pw[kSelPer], pv[kSelPer], sa[kSelPer];  // inclusive prefixes (w, v) and suffix (a) in the thread
  double tw = 0.0, tv = 0.0, ta = 0.0;
  if (wg < nwa) {
    pw[0] = tw = cw[e0];
    pv[0] = tv = cv[e0];
#pragma unroll
    for (int k = 1; k < kSelPer; ++k) {
      if (k >= E) break;
      pw[k] = tw = pw[k - 1] + cw[e0 + k];
      pv[k] = tv = pv[k - 1] + cv[e0 + k];
    }
#pragma unroll
    for (int k = kSelPer - 1; k >= 0; --k) {
      if (k >= E) continue;
      sa[k] = k + 1 < E ? sa[k + 1 < kSelPer ? k + 1 : k] + ca[e0 + k] : ca[e0 + k];
    }
    ta = sa[0];
  }
  double wex, vex, asuf;
  scan3_active(tw, tv, ta, nwa, g, wg, wex, vex, asuf, scan_sh[g]);
  int ff = M;  // first compacted entry whose lower edge fails phi < r^2
  double Wlo = 0.0, Vlo = 0.0, Ahi = 0.0;
  if (wg < nwa) {
    Wlo = W0 + wex;  // W below this thread's first entry
    Vlo = V0 + vex;
    Ahi = A0 + asuf;  // A after this thread's last entry
#pragma unroll
    for (int k = kSelPer - 1; k >= 0; --k) {
      const int e = e0 + k;
      if (k >= E || e >= M) continue;
      // edges past +inf are NaN bit patterns and fail
      const unsigned Tbits = base | ((unsigned)cb[e] << shift);
      const double Tb = (double)__uint_as_float(Tbits);
      const double Wb = k > 0 ? Wlo + pw[k > 0 ? k - 1 : 0] : Wlo;
      const double Ain = Ahi + sa[k];
      const double phi = nonneg_positive(Ain) ? fma(Tb * Tb, Ain, Wb) : Wb;
      if ((Tbits & 0x7fffffffu) > 0x7f800000u || !nonneg_less(phi, r2)) ff = e;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ff = min(ff, __shfl_xor_sync(0xffffffffu, ff, o));
  if (lane == 0) s_ff[g][wg] = ff;
  group_sync(g);
  ff = M;
#pragma unroll
  for (int q = 0; q < kSelWarps; ++q) ff = min(ff, s_ff[g][q]);
  // 3. the chosen bucket and the sums below / after it
  const int sel = ff > 0 ? ff - 1 : 0;
  if (wg >= nwa || sel < e0 || sel >= e0 + E) return;
  const int k = sel - e0;
  // the chosen entry's in-thread sums (static register indices)
  double pw_b = 0.0, pv_b = 0.0, sa_a = 0.0;
  const double lw_k = cw[sel], lv_k = cv[sel];
#pragma unroll
  for (int kk = 0; kk < kSelPer; ++kk) {
    if (kk != k) continue;
    if (kk > 0) { pw_b = pw[kk > 0 ? kk - 1 : 0]; pv_b = pv[kk > 0 ? kk - 1 : 0]; }
    if (kk + 1 < kSelPer) sa_a = sa[kk + 1 < kSelPer ? kk + 1 : kk];
  }
  const double Wb = k > 0 ? Wlo + pw_b : Wlo;
  const double Vb = k > 0 ? Vlo + pv_b : Vlo;
  const double Aout = k + 1 < E ? Ahi + sa_a : Ahi;
  if (ff == 0 && cb[0] > 0) {
    // the first nonempty bucket's edge already fails and it lies above the
    // range's start: the crossing is in the empty buckets below it, and no
    // item of the range is clipped
    s->g_prefix[slot] = base | ((unsigned)(cb[0] - 1) << shift);
    gap_final(s, slot, Wb, Vb, Ahi + sa[0], r2, s_r[g]);
    return;
  }
  // (ff = 0 with the first bucket at the range's start: its own edge failed
  // by rounding, and it is taken, as in a dense selection)
  s->g_W[slot] = Wb;
  s->g_V[slot] = Vb;
  s->g_A[slot] = Aout;
  s->g_prefix[slot] = base | ((unsigned)cb[sel] << shift);
  // the items of the last digit's bucket share one float key: clipped
  if (pass == 2) gap_final(s, slot, Wb + lw_k, Vb + lv_k, Aout, r2, s_r[g]);
}

__device__ void decide(Scalars *s, double *trace);
__device__ void pw_candidate(Scalars *s, int c);

template <typename T>
__global__ void __launch_bounds__(kGapThreads, 1) k_gap_pass(Problem<T> P, State<T> S, int pass, int s_begin,
                                                          int s_end, int when_restart, int with_decide) {
  extern __shared__ __align__(16) double hist[];  // [slots][3][kGapBuckets]
  __shared__ double s_gin[kGapSlots][4];
  __shared__ unsigned s_gpref[kGapSlots];
  Scalars *sc = S.s;
  if (when_restart ? !sc->restart : !sc->do_gap) return;  // uniform over the grid
  // a launch covers slots s_begin + q, q < 2; per-slot state by q (registers)
  bool act[2];
  for (int q = 0; q < 2; ++q) act[q] = s_begin + q < s_end && sc->g_active[s_begin + q];
  // every slot finished in an earlier pass (its decision, if any, was taken
  // there); pass 0 still runs the decision when no slot was active at all
  if (!act[0] && !act[1] && (pass > 0 || !with_decide)) return;
  const int ns = s_end - s_begin;
  int shift, nb, pshift;
  gap_digits(pass, shift, nb, pshift);
  for (int e = threadIdx.x; e < ns * 3 * kGapBuckets; e += blockDim.x) hist[e] = 0.0;
  if (threadIdx.x < kGapSlots) {
    const int q = threadIdx.x;
    // the slot's selection state, read once here rather than by the last
    // CTA's selection after the ticket
    s_gin[q][0] = sc->g_W[q];
    s_gin[q][1] = sc->g_V[q];
    s_gin[q][2] = sc->g_A[q];
    s_gin[q][3] = sc->g_r2[q];
    s_gpref[q] = sc->g_prefix[q];
  }
  // Algorithm 3 for both candidates, beside this CTA's items (lanes 0 of
  // warps 1 and 3: distinct sub-partitions)
  if (pass == 0 && with_decide && blockIdx.x == gridDim.x - 1 && (threadIdx.x == 32 || threadIdx.x == 96))
    pw_candidate(sc, threadIdx.x == 32 ? 0 : 1);
  __syncthreads();
  const int N = P.n + P.m;
  unsigned pref[2];
  double om[2], inv_om[2], ainf[2];
  int slot[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    slot[q] = act[q] ? s_begin + q : 0;
    pref[q] = pass == 0 ? 0u : s_gpref[slot[q]] >> pshift;
    om[q] = sc->g_omega[slot[q]];
    inv_om[q] = sc->g_inv_omega[slot[q]];
    ainf[q] = 0.0;
  }
  const int stride = gridDim.x * blockDim.x;
  if (pass == 0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!act[q]) continue;
        const GapItem it = gap_item<T>(P, S, sc, slot[q], i, om[q], inv_om[q]);
        S.gkeys[(size_t)slot[q] * N + i] = it.key;
        if (it.key == kKeyNone) continue;
        if (it.key == kKeyInf) { ainf[q] += it.a; continue; }
        const int b = (int)((it.key >> shift) & (unsigned)(nb - 1));
        double *h = hist + (size_t)q * 3 * kGapBuckets;
        atomicAdd(h + b, it.w);
        atomicAdd(h + kGapBuckets + b, it.v);
        atomicAdd(h + 2 * kGapBuckets + b, it.a);
      }
    }
  } else {
    // later digits: only the items of the selected bucket; the keys of
    // kKeyBatch strided items are loaded together (the loop is bound by
    // their latency, not by the few items that match)
    constexpr int kKeyBatch = 4;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += kKeyBatch * stride) {
      unsigned key[kKeyBatch][2];
#pragma unroll
      for (int u = 0; u < kKeyBatch; ++u) {
        const int i = i0 + u * stride;
#pragma unroll
        for (int q = 0; q < 2; ++q) key[u][q] = (act[q] && i < N) ? S.gkeys[(size_t)slot[q] * N + i] : kKeyNone;
      }
#pragma unroll
      for (int u = 0; u < kKeyBatch; ++u) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const unsigned k = key[u][q];
          if (k >= kKeyInf || (k >> pshift) != pref[q]) continue;  // none, inf, other bucket
          const GapItem it = gap_item<T>(P, S, sc, slot[q], i0 + u * stride, om[q], inv_om[q]);
          const int b = (int)((it.key >> shift) & (unsigned)(nb - 1));
          double *h = hist + (size_t)q * 3 * kGapBuckets;
          atomicAdd(h + b, it.w);
          atomicAdd(h + kGapBuckets + b, it.v);
          atomicAdd(h + 2 * kGapBuckets + b, it.a);
        }
      }
    }
  }
  if (pass == 0) {  // unbounded directions: their a goes to the +inf bucket, one atomic per warp
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!act[q]) continue;
      double t = ainf[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if ((threadIdx.x & 31) == 0 && nonneg_positive(t))
        atomicAdd(hist + (size_t)q * 3 * kGapBuckets + 2 * kGapBuckets + (kKeyInf >> 21), t);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!act[q]) continue;
    const double *h = hist + (size_t)q * 3 * kGapBuckets;
    double *gh = S.ghist + (size_t)slot[q] * kGapBuckets * 3;
    unsigned *gm = S.gmask + (size_t)slot[q] * (kGapBuckets / 32);
    // nb is a multiple of the CTA size: every lane takes each ballot
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double hw = h[b], hv = h[kGapBuckets + b], ha = h[2 * kGapBuckets + b];
      // bit tests, no float64 compares
      if (__double_as_longlong(hw) != 0ll) atomicAdd(gh + b, hw);
      if (__double_as_longlong(hv) != 0ll) atomicAdd(gh + kGapBuckets + b, hv);
      if (__double_as_longlong(ha) != 0ll) atomicAdd(gh + 2 * kGapBuckets + b, ha);
      const unsigned bal = __ballot_sync(0xffffffffu, !bucket_empty(hw, hv, ha));
      if ((threadIdx.x & 31) == 0 && bal) atomicOr(gm + (b >> 5), bal);
    }
  }
  if (last_block(S.tickets + kTicketGap)) {
    // the active slots, one per selection group (group g = warp parity)
    const int g = (threadIdx.x >> 5) & 1;
    const int q = (act[0] && act[1]) ? g : (act[1] ? 1 : 0);
    if (act[q] && (g == 0 || (act[0] && act[1]))) {
      const int s = slot[q];
      gap_select(sc, s, pass, S.ghist + (size_t)s * kGapBuckets * 3, S.gmask + (size_t)s * (kGapBuckets / 32),
                 hist + (size_t)g * kSelSmem, s_gin[s], s_gpref[s], g);
    }
    __syncthreads();
    // the restart decision as soon as the candidates' gaps are known (the
    // pass in which the last of them finished; later passes return at once)
    if (with_decide && threadIdx.x == 0) {
      bool done = true;
      for (int s = s_begin; s < s_end; ++s) done = done && !sc->g_active[s];
      if (done) decide(sc, S.trace);
    }
  }
}

// --------------------------------------------------- restart (Section 3.2)

// Algorithm 3 for candidate c (Delta = the candidate's distances to
// z^{n,0}), should the restart take it: the new primal weight, its
// reciprocal and the radius^2 of the restart point's gap under it.  Computed
// early in the candidates' first gap pass (a float64 square root, logarithm
// or exponential takes several hundred cycles on this part), so that the
// decision itself is a choice.
__device__ void pw_candidate(Scalars *s, int c) {
  if (c == 1 && !(s->sum_eta > 0.0)) return;
  const double dx2 = s->cand_dx2[c], dy2 = s->cand_dy2[c];
  const double Dx = sqrt(dx2), Dy = sqrt(dy2);
  double om = s->omega;
  if (s->pw_update && Dx > s->eps_zero && Dy > s->eps_zero)
    om = exp(s->pw_theta * log(Dy / Dx) + (1.0 - s->pw_theta) * log(om));
  s->pw_omega[c] = om;
  s->pw_inv[c] = 1.0 / om;
  s->pw_r2[c] = om * dx2 + dy2 / om;
}

// GetRestartCandidate, criteria (i)-(iii) and Algorithm 3.  One thread (of
// the last CTA of the candidates' final gap pass).
__device__ void decide(Scalars *s, double *trace) {
  if (!s->do_gap) return;
  const double mu_c = s->mu[0];
  const double mu_a = s->sum_eta > 0.0 ? s->mu[1] : INFINITY;
  // restart_to_current = 0: the average whenever there is one (Appendix C.2)
  const int cand = s->restart_to_current ? (mu_c < mu_a ? 0 : 1) : (s->sum_eta > 0.0 ? 1 : 0);
  const double muc = cand == 0 ? mu_c : mu_a;
  int restart = 0;
  if (muc <= s->beta_suff * s->mu0) restart = 1;
  else if (muc <= s->beta_nec * s->mu0 && muc > s->muc_prev) restart = 1;
  else if ((double)s->t >= s->beta_art * (double)s->k) restart = 1;
  s->muc_prev = muc;
  s->cand = cand;
  s->restart = restart;
  double *rec = trace + (size_t)(s->trace_n % kTraceCap) * kTraceLen;
  s->trace_n += 1;
  rec[0] = (double)s->k;
  rec[1] = (double)s->t;
  rec[2] = mu_c;
  rec[3] = mu_a;
  rec[4] = s->mu0;
  rec[5] = (double)cand;
  rec[6] = (double)restart;
  rec[7] = s->omega;
  rec[8] = sqrt(s->g_r2[0]);
  rec[9] = sqrt(s->g_r2[1]);
  rec[10] = s->kkt[0][5];
  rec[11] = s->kkt[0][6];
  rec[12] = s->kkt[0][7];
  rec[13] = s->kkt[1][5];
  rec[14] = s->kkt[1][6];
  rec[15] = s->kkt[1][7];
  if (!restart) return;
  // Algorithm 3 for the chosen candidate, computed by pw_candidate
  s->omega = s->pw_omega[cand];
  s->inv_omega = s->pw_inv[cand];
  s->tau = s->eta * s->inv_omega;
  s->sigma = s->eta * s->omega;
  rec[7] = s->omega;
  // slot 2: mu_n(z^{n+1,0}, z^{n,0}) under the new primal weight
  const double r2 = s->pw_r2[cand];
  s->g_r2[2] = r2;
  s->g_omega[2] = s->omega;
  s->g_inv_omega[2] = s->inv_omega;
  s->g_W[2] = s->g_V[2] = s->g_A[2] = 0.0;
  s->g_prefix[2] = 0u;
  s->g_active[2] = r2 > 0.0 ? 1 : 0;
  s->mu[2] = INFINITY;
  s->gval[2] = 0.0;
}

// z^{n+1,0} = candidate; current iterate = candidate; sums reset.
template <typename T>
__global__ void k_apply_restart(Problem<T> P, State<T> S) {
  const Scalars *sc = S.s;
  if (sc->vrestart) {  // no-restart mode: only the reference point of the next update moves
    const int cur = sc->cur, n = P.n, N = P.n + P.m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
      if (i < n) S.x0[i] = S.x[cur][i];
      else S.y0[i - n] = S.y[cur][i - n];
    }
    return;
  }
  if (!sc->restart) return;
  const int cur = sc->cur, cand = sc->cand;
  const double inv = sc->inv_avg;
  // to the average: y moves, and the stored K^T y no longer holds
  if (cand == 1 && blockIdx.x == 0 && threadIdx.x == 0) S.s->kty_valid = 0;
  const int n = P.n, N = P.n + P.m;
  T *x = S.x[cur], *xs = S.xs[cur], *y = S.y[cur], *ys = S.ys[cur], *Kx = S.Kx[cur];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const T v = cand == 0 ? x[i] : (T)((double)xs[i] * inv);
      x[i] = v;
      S.x0[i] = v;
      xs[i] = T(0);
    } else {
      const int r = i - n;
      const T v = cand == 0 ? y[r] : (T)((double)ys[r] * inv);
      y[r] = v;
      S.y0[r] = v;
      ys[r] = T(0);
      if (cand == 1) Kx[r] = (T)((double)S.Kxbar[r] * inv);
    }
  }
}

__device__ void finish_state(Scalars *s, cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_inner,
                             int has_inner, int has_cond, cudaGraphConditionalHandle h_rs, int has_rs);

// After the restart point's gap (slot 2): mu_0 of the new outer loop, empty
// running sums, the restart counted.
__device__ __forceinline__ void restart_done(Scalars *s) {
  if (s->restart) {
    s->mu0 = s->mu[2];
    s->sum_eta = 0.0;
    s->t = 0;
    s->muc_prev = INFINITY;
    s->restarts += 1;
    s->restart = 0;
  }
  s->vrestart = 0;
}

// End of an evaluation: the loop conditions, and (has_rs) the condition of
// the graph's restart branch (apply restart, restart point's gap,
// k_restart_done), which then follows; without has_rs that branch already
// ran and its book-keeping happens here.  (The Algorithm 2 factors of the
// next chunk are filled by k_eval_rows.)
__global__ void k_finish(Scalars *s, cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_inner,
                         int has_inner, int has_cond = 1, cudaGraphConditionalHandle h_rs = 0, int has_rs = 0) {
  if (threadIdx.x == 0) finish_state(s, h_outer, h_inner, has_inner, has_cond, h_rs, has_rs);
}

__global__ void k_restart_done(Scalars *s) {
  if (threadIdx.x == 0) restart_done(s);
}

__device__ void finish_state(Scalars *s, cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_inner,
                             int has_inner, int has_cond, cudaGraphConditionalHandle h_rs, int has_rs) {
  if (has_rs) cudaGraphSetConditional(h_rs, (s->restart || s->vrestart) ? 1u : 0u);
  else restart_done(s);
  s->do_gap = 0;
  s->chunk_acc = 0;
  if (s->err) s->status = kWaitTimeout;
  if (s->status == kRunning && time_up(s)) s->status = kTimeLimit;
  const bool run = s->status == kRunning;
  if (has_cond) cudaGraphSetConditional(h_outer, run ? 1u : 0u);
  if (has_cond && has_inner) cudaGraphSetConditional(h_inner, run ? 1u : 0u);
}

// ------------------------------------------------------------- set-up / out

// Norms of the problem data: ||c||, ||q|| (original), ||c~||, ||q~|| (scaled)
// -> InitializePrimalWeight (Section 3.3) times primal_importance.
template <typename T>
__global__ void k_problem_norms(Problem<T> P, Scalars *s, double primal_importance, double *part) {
  __shared__ double red[4 * (kThreads / 32)];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int N = P.n + P.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < P.n) {
      acc[0] += P.c[i] * P.c[i];
      const double cs = (double)P.cs[i];
      acc[2] += cs * cs;
    } else {
      const int r = i - P.n;
      acc[1] += P.q[r] * P.q[r];
      const double qs = (double)P.qs[r];
      acc[3] += qs * qs;
    }
  }
  block_sum<4>(acc, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 4; ++a) part[4 * blockIdx.x + a] = acc[a];
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    // tickets live after the 4*gridDim partials
    unsigned *ticket = reinterpret_cast<unsigned *>(part + 4 * gridDim.x);
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    if (s_last) *ticket = 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[4];
  sum_partials<4>(part, gridDim.x, 4, tot, red);
  if (threadIdx.x == 0) {
    s->cnorm = sqrt(tot[0]);
    s->qnorm = sqrt(tot[1]);
    const double nc = sqrt(tot[2]), nq = sqrt(tot[3]);
    const double w = (nc > s->eps_zero && nq > s->eps_zero) ? nc / nq : 1.0;
    s->omega = w * primal_importance;
  }
}

// Start point z^{0,0} (scaled, projected onto X x Y), sums, restart point.
template <typename T>
__global__ void k_init_point(Problem<T> P, State<T> S, const double *x0, const double *y0) {
  const int n = P.n, N = P.n + P.m;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // barrier counter of the persistent kernel
    S.tickets[kTicketBar] = 0u;
    S.tickets[kTicketBar + 1] = 0u;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double v = x0 ? x0[i] / P.D2[i] : 0.0;
      const T x = clampv<T>((T)v, P.ls[i], P.us[i]);
      S.x[0][i] = x;
      S.x0[i] = x;
      S.xs[0][i] = T(0);
      S.xs[1][i] = T(0);
    } else {
      const int r = i - n;
      const double v = y0 ? y0[r] / P.D1[r] : 0.0;
      const T lo = P.ylos[r];
      const T y = (T)v > lo ? (T)v : lo;
      S.y[0][r] = y;
      S.y0[r] = y;
      S.ys[0][r] = T(0);
      S.ys[1][r] = T(0);
    }
  }
}

// Plain row sums out[i] = sum_k A_ik v[col_k] over the row-block schedule.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_spmv(Mat<T> A, const T *v, T *out) {
  extern __shared__ __align__(16) char sm[];
  const T *const vec[1] = {v};
  double none[1] = {0.0};
  spmv_warp<T, 1>(A, vec, sm, none, [&](int i, const T(&s)[1], double(&)[1]) { out[i] = s[0]; });
}

__global__ void k_init_scalars(Scalars *s, ScalarInit in) {
  s->eta = in.eta0;
  s->kty_valid = 0;
  if (in.omega0 > 0.0) s->omega = in.omega0;  // else omega^0 as set by k_problem_norms
  s->inv_omega = 1.0 / s->omega;
  s->const_step = in.const_step;
  s->tau = in.eta0 * s->inv_omega;
  s->sigma = in.eta0 * s->omega;
  s->sum_eta = 0.0;
  s->mu0 = INFINITY;
  s->muc_prev = INFINITY;
  s->inv_avg = 0.0;
  s->rel_tol = in.tol_dev ? *in.tol_dev : in.rel_tol;
  s->beta_suff = in.beta_suff;
  s->beta_nec = in.beta_nec;
  s->beta_art = in.beta_art;
  s->pw_theta = in.pw_theta;
  s->eps_zero = in.eps_zero;
  s->k = s->t = s->attempts = s->restarts = 0;
  s->iter_limit = in.lim_dev ? in.lim_dev[0] : in.iter_limit;
  s->attempt_limit = in.lim_dev ? in.lim_dev[1] : in.attempt_limit;
  s->time_limit_ns = in.lim_dev ? (unsigned long long)in.lim_dev[2] : in.time_limit_ns;
  s->t0_ns = global_timer_ns();
  s->t_end_ns = 0;
  s->cur = 0;
  s->chunk_acc = 0;
  s->eval_every = in.eval_every;
  s->status = kRunning;
  s->ret_which = 0;
  s->phase = 0;
  s->do_gap = 0;
  s->restart = 0;
  s->cand = 0;
  s->adaptive_restart = in.adaptive_restart;
  s->pw_update = in.pw_update;
  s->err = 0;
  s->trace_n = 0;
  for (int a = 0; a < kGapSlots; ++a) { s->g_active[a] = 0; s->mu[a] = INFINITY; }
  s->restart_to_current = in.restart_to_current;
  s->vrestart = 0;
  s->k_virt = 0;
  s->mp = in.mp;
  s->mp_trial = 0;
  s->mp_bf = in.mp_breaking;
  s->mp_df = in.mp_downscaling;
  s->mp_ic = in.mp_interpolation;
  s->mp_eta_k = in.eta0;
  s->mp_theta = 1.0;  // theta_0 (no earlier step)
  s->mp_eh = s->mp_eta_k + s->mp_ic * (sqrt(1.0 + s->mp_theta) - 1.0) * s->mp_eta_k;
  s->mp_th = s->mp_eta_k / s->mp_eh;
  s->stall_best = INFINITY;
  s->stall_count = 0;
  s->stall_evals = in.stall_evals;
  s->wait_ns = in.wait_ns ? in.wait_ns : kBarrierTimeoutNs;
  s->wait_extra = in.wait_extra;
}

// Returned point in the original space: x = D2 x~, y = D1 y~.
template <typename T>
__global__ void k_output(Problem<T> P, State<T> S) {
  Scalars *sc = S.s;
  const int cur = sc->cur, which = sc->ret_which;
  const double inv = sc->inv_avg;
  const int n = P.n, N = P.n + P.m;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->t_end_ns = global_timer_ns();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double x = which == 0 ? (double)S.x[cur][i] : (double)S.xs[cur][i] * inv;
      S.xo[i] = P.D2[i] * x;
    } else {
      const int r = i - n;
      const double y = which == 0 ? (double)S.y[cur][r] : (double)S.ys[cur][r] * inv;
      S.yo[r] = P.D1[r] * y;
    }
  }
}

// ------------------------------------------------------- graph construction

// histogram of `ns` slots; the selection also needs room for 2049 suffix sums
static size_t gap_smem(int ns) {
  const size_t hist = (size_t)3 * ns * kGapBuckets, sel = (size_t)ns * kSelSmem;
  return sizeof(double) * ((hist > sel ? hist : sel) + 8);
}

template <typename T>
static size_t spmv_smem(int nv) {
  return spmv_smem_bytes<T>(nv);
}

template <typename T>
cudaError_t set_kernel_attributes() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_primal<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_dual<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_eval_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(2)))) return e;
  if ((e = cudaFuncSetAttribute(k_eval_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_spmv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_mp_primal<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_mp_kx<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  if ((e = cudaFuncSetAttribute(k_mp_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_smem<T>(1)))) return e;
  const int gsm = (int)gap_smem(2);
  if ((e = cudaFuncSetAttribute(k_gap_pass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm))) return e;
  return cudaSuccess;
}

template <typename T>
static void launch_gap(const Problem<T> &P, const State<T> &S, int s_begin, int s_end, int when_restart,
                       int grid, cudaStream_t st, int with_decide = 0) {
  const size_t smem = gap_smem(s_end - s_begin);
  for (int pass = 0; pass < 3; ++pass)
    k_gap_pass<T><<<grid, kGapThreads, smem, st>>>(P, S, pass, s_begin, s_end, when_restart, with_decide);
}

template <typename T>
cudaError_t launch_gap_slots(const Problem<T> &P, const State<T> &S, int s_begin, int s_end, int when_restart,
                             int grid, cudaStream_t st) {
  launch_gap<T>(P, S, s_begin, s_end, when_restart, grid, st);
  return cudaGetLastError();
}

// One trial of the Malitsky-Pock line search (k_mp_test sets h when has_cond).
template <typename T>
static void launch_mp_trial(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                            cudaGraphConditionalHandle h, int has_cond, cudaStream_t st) {
  const int gd = K.nblocks > 0 ? K.nblocks : 1;  // part_d holds 2 K.nblocks entries
  if (KT.nblocks > 0) k_mp_primal<T><<<KT.nblocks, kThreads, spmv_smem<T>(1), st>>>(KT, P, S);
  if (K.nblocks > 0) k_mp_kx<T><<<K.nblocks, kThreads, spmv_smem<T>(1), st>>>(K, S);
  k_mp_dual<T><<<gd, kThreads, 0, st>>>(P, S);
  if (KT.nblocks > 0) k_mp_cols<T><<<KT.nblocks, kThreads, spmv_smem<T>(1), st>>>(KT, S);
  k_mp_test<T><<<1, kThreads, 0, st>>>(KT, S, KT.nblocks, gd, h, has_cond);
}

template <typename T>
cudaError_t launch_step_pair(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                             cudaStream_t st) {
  launch_attempt<T>(K, KT, P, S, 0, 0, st);
  return cudaGetLastError();
}
template cudaError_t launch_step_pair<double>(const Mat<double> &, const Mat<double> &, const Problem<double> &,
                                              const State<double> &, cudaStream_t);
template cudaError_t launch_step_pair<float>(const Mat<float> &, const Mat<float> &, const Problem<float> &,
                                             const State<float> &, cudaStream_t);

template <typename T>
__global__ void k_pow_fill(T *v, int n) {
  const T val = (T)(1.0 / sqrt((double)n));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = val;
}

// ||u||_2 by one CTA in fixed order -> nrm[0]; v = u / ||u|| by the grid.
template <typename T>
__global__ void __launch_bounds__(1024) k_pow_norm(const T *u, int n, double *nrm) {
  __shared__ double red[1024 / 32];
  double a[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[0] += (double)u[i] * (double)u[i];
  block_sum<1>(a, red);
  if (threadIdx.x == 0) nrm[0] = sqrt(a[0]);
}

template <typename T>
__global__ void k_pow_scale(const T *u, int n, const double *nrm, T *v) {
  const double s = nrm[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = s > 0.0 ? (T)((double)u[i] / s) : u[i];
}

template <typename T>
cudaError_t power_norm(const Mat<T> &A, const Mat<T> &AT, int iters, T *v, T *w, T *u, double *nrm,
                       cudaStream_t st, double *out) {
  const int n = A.cols;
  const int g = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
  k_pow_fill<T><<<g, 256, 0, st>>>(v, n);
  for (int it = 0; it < iters; ++it) {
    launch_spmv<T>(A, v, w, st);
    launch_spmv<T>(AT, w, u, st);
    k_pow_norm<T><<<1, 1024, 0, st>>>(u, n, nrm);
    k_pow_scale<T><<<g, 256, 0, st>>>(u, n, nrm, v);
  }
  cudaError_t e;
  double h = 0.0;
  if ((e = cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  *out = sqrt(h);
  return cudaGetLastError();
}
template cudaError_t power_norm<double>(const Mat<double> &, const Mat<double> &, int, double *, double *,
                                        double *, double *, cudaStream_t, double *);
template cudaError_t power_norm<float>(const Mat<float> &, const Mat<float> &, int, float *, float *, float *,
                                       double *, cudaStream_t, double *);

template <typename T>
void launch_spmv(const Mat<T> &A, const T *v, T *out, cudaStream_t st) {
  if (A.nblocks > 0) k_spmv<T><<<A.nblocks, kThreads, spmv_smem<T>(1), st>>>(A, v, out);
}

template <typename T>
void launch_problem_norms(const Problem<T> &P, Scalars *s, double primal_importance, double *part,
                          int grid, cudaStream_t st) {
  k_problem_norms<T><<<grid, kThreads, 0, st>>>(P, s, primal_importance, part);
}

template <typename T>
void launch_init(const Problem<T> &P, const State<T> &S, const Mat<T> &K, const ScalarInit &in,
                 const double *x0, const double *y0, cudaStream_t st) {
  k_init_scalars<<<1, 1, 0, st>>>(S.s, in);
  const int N = P.n + P.m;
  k_init_point<T><<<(N + 255) / 256, 256, 0, st>>>(P, S, x0, y0);
  launch_spmv<T>(K, S.x[0], S.Kx[0], st);
}

template <typename T>
void launch_eval(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S, cudaStream_t st) {
  if (KT.nblocks > 0) k_eval_cols<T><<<KT.nblocks, kThreads, spmv_smem<T>(2), st>>>(K, KT, P, S);
  k_eval_rows<T><<<K.nblocks, kThreads, spmv_smem<T>(1), st>>>(K, KT, P, S);
}

// The evaluation with its column kernel on a side stream, so that the two
// kernels run concurrently (their float64 pipes are each about half busy);
// `st` waits for both.
template <typename T>
static void launch_eval_fork(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                             cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  cudaEventRecord(ev_fork, st);
  cudaStreamWaitEvent(side, ev_fork, 0);
  if (KT.nblocks > 0) k_eval_cols<T><<<KT.nblocks, kThreads, spmv_smem<T>(2), side>>>(K, KT, P, S);
  k_eval_rows<T><<<K.nblocks, kThreads, spmv_smem<T>(1), st>>>(K, KT, P, S);
  cudaEventRecord(ev_join, side);
  cudaStreamWaitEvent(st, ev_join, 0);
}

template <typename T>
void launch_output(const Problem<T> &P, const State<T> &S, cudaStream_t st) {
  const int N = P.n + P.m;
  k_output<T><<<(N + 255) / 256, 256, 0, st>>>(P, S);
}

// The graph that `st` is capturing into.
static cudaError_t capture_graph(cudaStream_t st, cudaGraph_t *g) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps;
  size_t ndeps;
  return cudaStreamGetCaptureInfo(st, &cs, nullptr, g, &deps, nullptr, &ndeps);
}

// Appends a conditional WHILE node on handle h (created in the capturing
// graph) after everything captured so far on `st`; returns its body graph.
static cudaError_t add_cond(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            cudaGraph_t *body) {
  cudaError_t e;
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t *deps;
  size_t ndeps;
  if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps))) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p))) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// IF (restart or virtual restart) { apply restart, gap of the restart point
// (slot 2), restart book-keeping }, captured on st4 into the branch's body.
template <typename T>
static cudaError_t add_restart_branch(const Problem<T> &P, const State<T> &S, int gap_grid,
                                      cudaGraphConditionalHandle h_rs, cudaStream_t st2, cudaStream_t st4) {
  cudaGraph_t body = nullptr;
  cudaError_t e = add_cond(st2, h_rs, cudaGraphCondTypeIf, &body);
  if (!e) e = cudaStreamBeginCaptureToGraph(st4, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e) return e;
  const int N = P.n + P.m;
  k_apply_restart<T><<<(N + 255) / 256, 256, 0, st4>>>(P, S);
  launch_gap<T>(P, S, 2, 3, 1, gap_grid, st4);
  k_restart_done<<<1, 32, 0, st4>>>(S.s);
  cudaGraph_t tmp;
  cudaError_t e2 = cudaStreamEndCapture(st4, &tmp);
  return e2;
}

// The whole solve as one graph:
//   norms, init, K x0, evaluation (termination check at the start), finish
//   WHILE running:
//     WHILE chunk not done: primal, dual (+ accept)
//     evaluation, gap (slots 0,1), decide, apply restart, gap (slot 2), finish
//   output
// Every loop is bounded: each inner pass makes one step attempt and the
// accept kernel stops the inner loop at attempt_limit; the evaluation turns
// the status to a limit once k or the attempts reach their limits, and the
// outer condition is the status.
template <typename T>
cudaError_t build_solve_graph(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                              const State<T> &S, const ScalarInit &in, double primal_importance, double *norm_part,
                              const double *x0_dev, const double *y0_dev, int gap_grid, const PersistGeo &pg,
                              const PersistGeo &pe, cudaStream_t st, cudaStream_t st2, cudaStream_t st3, cudaStream_t st4,
                              cudaGraphExec_t *exec) {
  cudaError_t e;
  cudaGraph_t graph = nullptr;
  *exec = nullptr;
  // fork / join of the evaluation's two kernels inside the loop body
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if ((e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming))) return e;
  if ((e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming))) {
    cudaEventDestroy(ev_fork);
    return e;
  }
  struct EventPair {
    cudaEvent_t a, b;
    ~EventPair() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } events{ev_fork, ev_join};
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal))) return e;
  const int N = P.n + P.m;
  launch_problem_norms<T>(P, S.s, primal_importance, norm_part, 152, st);
  k_init_scalars<<<1, 1, 0, st>>>(S.s, in);
  k_init_point<T><<<(N + 255) / 256, 256, 0, st>>>(P, S, x0_dev, y0_dev);
  launch_spmv<T>(K, S.x[0], S.Kx[0], st);
  launch_eval<T>(K, KT, P, S, st);
  cudaGraphConditionalHandle h_outer = 0, h_inner = 0, h_rs = 0;
  cudaGraph_t g = nullptr, body_outer = nullptr, body_inner = nullptr;
  e = capture_graph(st, &g);
  if (!e) e = cudaGraphConditionalHandleCreate(&h_outer, g, 0u, cudaGraphCondAssignDefault);
  if (!e) {
    k_finish<<<1, 64, 0, st>>>(S.s, h_outer, h_outer, 0);  // loop entry decided by the check at the start
    e = add_cond(st, h_outer, cudaGraphCondTypeWhile, &body_outer);
  }
  // the restart branch's condition: set by k_finish in every evaluation
  if (!e) e = cudaGraphConditionalHandleCreate(&h_rs, body_outer, 0u, 0u);
  if (!e) e = cudaStreamBeginCaptureToGraph(st2, body_outer, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (!e && pg.grid > 0) {
    // one persistent cooperative kernel per chunk of step attempts
    e = launch_persist<T>(K, KT, P, S, pg, st2);
    if (!e) {
      // the evaluation: one persistent launch on the step kernel's grid
      // (float64), else the column and row kernels on two streams
      if (pe.grid > 0)
        e = launch_eval_persist<T>(K, KT, KTb, P, S, pe, st2);
      else
        launch_eval_fork<T>(K, KT, P, S, st2, st3, ev_fork, ev_join);
    }
    if (!e) {
      launch_gap<T>(P, S, 0, 2, 0, gap_grid, st2, 1);  // with the restart decision
      k_finish<<<1, 64, 0, st2>>>(S.s, h_outer, h_outer, 0, 1, h_rs, 1);
      e = add_restart_branch<T>(P, S, gap_grid, h_rs, st2, st4);
    }
    cudaGraph_t tmp2;
    cudaError_t e2 = cudaStreamEndCapture(st2, &tmp2);
    if (!e) e = e2;
  } else if (!e) {
    e = cudaGraphConditionalHandleCreate(&h_inner, body_outer, 1u, cudaGraphCondAssignDefault);
    if (!e) e = add_cond(st2, h_inner, cudaGraphCondTypeWhile, &body_inner);
    if (!e) e = cudaStreamBeginCaptureToGraph(st3, body_inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (!e) {
      if (in.mp) {
        launch_mp_trial<T>(K, KT, P, S, h_inner, 1, st3);
      } else {
        launch_attempt<T>(K, KT, P, S, h_inner, 1, st3);
      }
      cudaGraph_t tmp;
      e = cudaStreamEndCapture(st3, &tmp);
    }
    if (!e) {
      launch_eval_fork<T>(K, KT, P, S, st2, st3, ev_fork, ev_join);
      launch_gap<T>(P, S, 0, 2, 0, gap_grid, st2, 1);  // with the restart decision
      k_finish<<<1, 64, 0, st2>>>(S.s, h_outer, h_inner, 1, 1, h_rs, 1);
      e = add_restart_branch<T>(P, S, gap_grid, h_rs, st2, st4);
    }
    cudaGraph_t tmp2;
    cudaError_t e2 = cudaStreamEndCapture(st2, &tmp2);
    if (!e) e = e2;
  }
  launch_output<T>(P, S, st);
  cudaError_t e3 = cudaStreamEndCapture(st, &graph);
  if (!e) e = e3;
  if (!e) e = cudaGetLastError();
  if (!e) e = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

// Times the two step kernels of one attempt outside the graph: `reps`
// launches of k_primal then k_dual (no loop condition), each pair bracketed by
// CUDA events on `st`.  The attempts advance the iterate like a solve does.
template <typename T>
cudaError_t time_step_kernels(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                              int reps, cudaStream_t st, float *ms_primal, float *ms_dual) {
  cudaEvent_t e0, e1, e2;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0))) return e;
  if ((e = cudaEventCreate(&e1))) return e;
  if ((e = cudaEventCreate(&e2))) return e;
  double tp = 0.0, td = 0.0;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    if (K.slab_on) k_primal_slab<T><<<KT.slab_grid, kSlabThreads, 0, st>>>(KT, P, S);
    else if (KT.nblocks > 0) k_primal<T><<<KT.nblocks, kThreads, spmv_smem<T>(1), st>>>(KT, P, S);
    cudaEventRecord(e1, st);
    if (K.slab_on) k_dual_slab<T><<<K.slab_grid, kSlabThreads, 0, st>>>(K, KT, P, S, 0, 0);
    else k_dual<T><<<K.nblocks, kThreads, spmv_smem<T>(1), st>>>(K, KT, P, S, 0, 0);
    cudaEventRecord(e2, st);
    if ((e = cudaEventSynchronize(e2))) break;
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    tp += a;
    td += b;
  }
  if (!e) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  *ms_primal = (float)(tp / reps);
  *ms_dual = (float)(td / reps);
  return e;
}

template cudaError_t time_step_kernels<double>(const Mat<double> &, const Mat<double> &, const Problem<double> &,
                                               const State<double> &, int, cudaStream_t, float *, float *);
template cudaError_t time_step_kernels<float>(const Mat<float> &, const Mat<float> &, const Problem<float> &,
                                              const State<float> &, int, cudaStream_t, float *, float *);
template cudaError_t launch_gap_slots<double>(const Problem<double> &, const State<double> &, int, int, int, int,
                                              cudaStream_t);
template cudaError_t launch_gap_slots<float>(const Problem<float> &, const State<float> &, int, int, int, int,
                                             cudaStream_t);
template cudaError_t set_kernel_attributes<double>();
template cudaError_t set_kernel_attributes<float>();
template void launch_spmv<double>(const Mat<double> &, const double *, double *, cudaStream_t);
template void launch_spmv<float>(const Mat<float> &, const float *, float *, cudaStream_t);
template void launch_problem_norms<double>(const Problem<double> &, Scalars *, double, double *, int, cudaStream_t);
template void launch_problem_norms<float>(const Problem<float> &, Scalars *, double, double *, int, cudaStream_t);
template void launch_init<double>(const Problem<double> &, const State<double> &, const Mat<double> &,
                                  const ScalarInit &, const double *, const double *, cudaStream_t);
template void launch_init<float>(const Problem<float> &, const State<float> &, const Mat<float> &,
                                 const ScalarInit &, const double *, const double *, cudaStream_t);
template void launch_eval<double>(const Mat<double> &, const Mat<double> &, const Problem<double> &,
                                  const State<double> &, cudaStream_t);
template void launch_eval<float>(const Mat<float> &, const Mat<float> &, const Problem<float> &,
                                 const State<float> &, cudaStream_t);
template void launch_output<double>(const Problem<double> &, const State<double> &, cudaStream_t);
template void launch_output<float>(const Problem<float> &, const State<float> &, cudaStream_t);
// The same solve with every kernel launched from a host loop (no graph):
// the state is read back after each step attempt and each evaluation.  Used
// where graph kernels cannot be observed individually (profilers) and as a
// fallback; the kernels and their order are those of the graph.
template <typename T>
cudaError_t run_stepped(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                        const ScalarInit &in, double primal_importance, double *norm_part, const double *x0_dev,
                        const double *y0_dev, int gap_grid, const PersistGeo &pg, cudaStream_t st, Scalars *host) {
  cudaError_t e;
  const int N = P.n + P.m;
  auto read = [&]() -> cudaError_t {
    cudaError_t e2 = cudaMemcpyAsync(host, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
    if (e2) return e2;
    return cudaStreamSynchronize(st);
  };
  launch_problem_norms<T>(P, S.s, primal_importance, norm_part, 152, st);
  k_init_scalars<<<1, 1, 0, st>>>(S.s, in);
  k_init_point<T><<<(N + 255) / 256, 256, 0, st>>>(P, S, x0_dev, y0_dev);
  launch_spmv<T>(K, S.x[0], S.Kx[0], st);
  launch_eval<T>(K, KT, P, S, st);
  k_finish<<<1, 64, 0, st>>>(S.s, 0, 0, 0, 0);
  if ((e = cudaGetLastError()) || (e = read())) return e;
  while (host->status == kRunning) {
    for (;;) {
      if (in.mp) {
        launch_mp_trial<T>(K, KT, P, S, 0, 0, st);
      } else if (pg.grid > 0) {
        if ((e = launch_persist<T>(K, KT, P, S, pg, st))) return e;
      } else {
        launch_attempt<T>(K, KT, P, S, 0, 0, st);
      }
      if ((e = cudaGetLastError()) || (e = read())) return e;
      const bool go = host->status == kRunning && !host->err && host->chunk_acc < host->eval_every &&
                      host->k < host->iter_limit && host->attempts < host->attempt_limit;
      if (!go) break;
    }
    launch_eval<T>(K, KT, P, S, st);
    launch_gap<T>(P, S, 0, 2, 0, gap_grid, st, 1);  // with the restart decision
    k_apply_restart<T><<<(N + 255) / 256, 256, 0, st>>>(P, S);
    launch_gap<T>(P, S, 2, 3, 1, gap_grid, st);
    k_finish<<<1, 64, 0, st>>>(S.s, 0, 0, 0, 0);
    if ((e = cudaGetLastError()) || (e = read())) return e;
  }
  launch_output<T>(P, S, st);
  if ((e = cudaGetLastError())) return e;
  return read();
}

template cudaError_t run_stepped<double>(const Mat<double> &, const Mat<double> &, const Problem<double> &,
                                         const State<double> &, const ScalarInit &, double, double *,
                                         const double *, const double *, int, const PersistGeo &, cudaStream_t, Scalars *);
template cudaError_t run_stepped<float>(const Mat<float> &, const Mat<float> &, const Problem<float> &,
                                        const State<float> &, const ScalarInit &, double, double *,
                                        const double *, const double *, int, const PersistGeo &, cudaStream_t, Scalars *);
template cudaError_t build_solve_graph<double>(const Mat<double> &, const Mat<double> &, const Mat<double> &,
                                               const Problem<double> &, const State<double> &, const ScalarInit &, double, double *,
                                               const double *, const double *, int, const PersistGeo &, const PersistGeo &, cudaStream_t,
                                               cudaStream_t, cudaStream_t, cudaStream_t, cudaGraphExec_t *);
template cudaError_t build_solve_graph<float>(const Mat<float> &, const Mat<float> &, const Mat<float> &,
                                              const Problem<float> &, const State<float> &, const ScalarInit &, double, double *,
                                              const double *, const double *, int, const PersistGeo &, const PersistGeo &, cudaStream_t,
                                              cudaStream_t, cudaStream_t, cudaStream_t, cudaGraphExec_t *);

}  // namespace pdlp
