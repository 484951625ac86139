// Unrolled PDHG (Eq. (3) with the step sizes of Algorithm 2 recorded and then
// held fixed, the primal weight fixed at its initial value, no restarts) and
// its hand-written adjoint.
//
// Forward map, step t (tau_t = eta_t / omega, sigma_t = eta_t * omega):
//   v_t     = x_t - tau_t (c - K^T y_t),           x_{t+1} = clip_[l,u](v_t)
//   w_t     = y_t + sigma_t (q - K (2 x_{t+1} - x_t)),  y_{t+1} = max(w_t, ylo)
// Reverse step, with xb, yb the adjoints of x_{t+1}, y_{t+1}:
//   h  = [w_t > ylo] yb
//   g  = [l < v_t < u] (xb - 2 sigma K^T h)
//   dq += sigma h,  dc -= tau g,  dK_ij += -sigma h_i (2 x_{t+1} - x_t)_j + tau y_t,i g_j
//   xb <- g + sigma K^T h,   yb <- h + tau K g
// all on the preconditioned problem; gradients with respect to the original
// data follow from c~ = D2 c, q~ = D1 q, K~_ij = D1_i K_ij D2_j with the
// preconditioner held fixed.  The reverse sweep runs segment by segment from
// the last checkpoint: it recomputes the segment's iterates (storing
// 2 x_{t+1} - x_t, y_t and the two projection masks per step), then walks
// back through it with one K^T and one K product per step.  The forward map
// runs in float64 or in float32 (then the recompute repeats its float32
// arithmetic); the adjoint and the gradients are float64.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "unroll.cuh"

namespace pdlp {

namespace {

constexpr int kEw = 256;  // elementwise CTA size

int ew_grid(int64_t n) { return (int)std::min<int64_t>((n + kEw - 1) / kEw, 152 * 16); }

// Resets the chunk counter and fills the step factors for the next segment.
__global__ void k_unr_segment(Scalars *s) {
  if (threadIdx.x == 0) {
    s->chunk_acc = 0;
    s->fac_k0 = s->k;
  }
  __syncthreads();
  fill_step_factors(s);
}

template <typename T>
__global__ void k_unr_out(int n, int m, const T *x, const T *y, const double *D2, const double *D1, double *xo,
                          double *yo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n)
      xo[i] = D2[i] * (double)x[i];
    else
      yo[i - n] = D1[i - n] * (double)y[i - n];
  }
}

// Forward primal half-step (the arithmetic of k_primal in type T) that also
// stores xe = 2 x' - x (float64) and the mask [l < v < u].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_unr_primal(Mat<T> KT, Problem<T> P, const T *x, const T *y, T *xn,
                                                         double *xe, uint8_t *mx, T tau) {
  extern __shared__ __align__(16) char sm[];
  double none[1] = {0.0};
  const T *const vec[1] = {y};
  spmv_warp<T, 1>(KT, vec, sm, none, [&](int j, const T(&g)[1], double(&)[1]) {
    const T xj = x[j];
    const T v = xj - tau * (P.cs[j] - g[0]);
    const T xp = clampv<T>(v, P.ls[j], P.us[j]);
    xn[j] = xp;
    xe[j] = 2.0 * (double)xp - (double)xj;
    mx[j] = (v > P.ls[j] && v < P.us[j]) ? 1 : 0;
  });
}

// Forward dual half-step (the arithmetic of k_dual in type T) that also
// stores y_t (float64) and the mask [w > ylo].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_unr_dual(Mat<T> K, Problem<T> P, const T *xn, const T *Kx, const T *y,
                                                       T *yn, T *Kxn, double *ys, uint8_t *my, T sigma) {
  extern __shared__ __align__(16) char sm[];
  double none[1] = {0.0};
  const T *const vec[1] = {xn};
  spmv_warp<T, 1>(K, vec, sm, none, [&](int i, const T(&s)[1], double(&)[1]) {
    const T kxn = s[0], kx = Kx[i], yi = y[i], lo = P.ylos[i];
    const T w = yi + sigma * (P.qs[i] - T(2) * kxn + kx);
    yn[i] = w > lo ? w : lo;
    Kxn[i] = kxn;
    ys[i] = (double)yi;
    my[i] = w > lo ? 1 : 0;
  });
}

__global__ void k_adj_h(int m, const double *yb, const uint8_t *my, double *h) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) h[i] = my[i] ? yb[i] : 0.0;
}

// Columns: K^T h, then g, dc and the new primal adjoint.
__global__ void __launch_bounds__(kThreads) k_adj_cols(Mat<double> KT, const double *h, const uint8_t *mx,
                                                       double *xb, double *g, double *dcs, double tau, double sigma) {
  extern __shared__ __align__(16) char sm[];
  double none[1] = {0.0};
  const double *const vec[1] = {h};
  spmv_warp<double, 1>(KT, vec, sm, none, [&](int j, const double(&s)[1], double(&)[1]) {
    const double kth = s[0];
    const double gg = mx[j] ? xb[j] - 2.0 * sigma * kth : 0.0;
    dcs[j] -= tau * gg;
    xb[j] = gg + sigma * kth;
    g[j] = gg;
  });
}

// Rows: K g, then dq and the new dual adjoint.
__global__ void __launch_bounds__(kThreads) k_adj_rows(Mat<double> K, const double *g, const double *h, double *yb,
                                                       double *dqs, double tau, double sigma) {
  extern __shared__ __align__(16) char sm[];
  double none[1] = {0.0};
  const double *const vec[1] = {g};
  spmv_warp<double, 1>(K, vec, sm, none, [&](int i, const double(&s)[1], double(&)[1]) {
    dqs[i] += sigma * h[i];
    yb[i] = h[i] + tau * s[0];
  });
}

__global__ void k_adj_dK(int64_t nnz, const int32_t *row, const int32_t *ci, const double *h, const double *ys,
                         const double *xe, const double *g, double *dKs, double tau, double sigma) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int i = row[k], j = ci[k];
    dKs[k] += -sigma * h[i] * xe[j] + tau * ys[i] * g[j];
  }
}

__global__ void k_adj_init(int n, int m, const double *gx, const double *gy, const double *D2, const double *D1,
                           double *xb, double *yb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n)
      xb[i] = D2[i] * gx[i];
    else
      yb[i - n] = gy ? D1[i - n] * gy[i - n] : 0.0;
  }
}

__global__ void k_adj_final(int n, int m, const double *D2, const double *D1, const double *dcs, const double *dqs,
                            double *dc, double *dq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n)
      dc[i] = D2[i] * dcs[i];
    else
      dq[i - n] = D1[i - n] * dqs[i - n];
  }
}

__global__ void k_adj_final_K(int64_t nnz, const int32_t *row, const int32_t *ci, const double *D1,
                              const double *D2, const double *dKs, double *dK) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    dK[k] = D1[row[k]] * D2[ci[k]] * dKs[k];
}

template <typename T>
size_t spmv_bytes() {
  return spmv_smem_bytes<T>(1);
}

}  // namespace

template <typename F>
cudaError_t unroll_forward(UnrollBuffers &U, const Mat<F> &K, const Mat<F> &KT, const Problem<F> &P,
                           const State<F> &S, const PersistGeo &pg, const ScalarInit &in, double primal_importance,
                           double *norm_part, int32_t T, int32_t ckpt, const double *x0, const double *y0,
                           cudaStream_t st) {
  cudaError_t e;
  const int n = P.n, m = P.m;
  U.ready = false;
  U.fp32 = sizeof(F) == 4;
  U.T = T;
  U.ckpt = ckpt;
  U.nseg = (T + ckpt - 1) / ckpt;
  F *ck = reinterpret_cast<F *>(U.ckpts.get(sizeof(F) * (size_t)U.nseg * (n + m)));
  U.eta = reinterpret_cast<double *>(U.etab.get(sizeof(double) * (size_t)T));
  double *outs = reinterpret_cast<double *>(U.outs.get(sizeof(double) * (size_t)(n + m)));
  if (!ck || !U.eta || !outs) return cudaErrorMemoryAllocation;
  U.xo = outs;
  U.yo = outs + n;
  State<F> S2 = S;
  S2.eta_log = U.eta;
  ScalarInit in2 = in;
  in2.iter_limit = T;
  in2.attempt_limit = 64ll * T + 64;  // Algorithm 2 accepts within a few attempts
  in2.time_limit_ns = 0ull;
  in2.lim_dev = nullptr;  // the unrolled map's own limits, not a refinement budget
  in2.eval_every = ckpt;
  in2.adaptive_restart = 0;
  in2.pw_update = 0;  // omega fixed over the unrolled map
  in2.mp = 0;
  launch_problem_norms<F>(P, S.s, primal_importance, norm_part, 152, st);
  launch_init<F>(P, S2, K, in2, x0, y0, st);
  if ((e = cudaGetLastError())) return e;
  Scalars h;
  int cur = 0;
  U.status = kRunning;
  for (int sg = 0; sg < U.nseg; ++sg) {
    F *slot = ck + (size_t)sg * (n + m);
    if ((e = cudaMemcpyAsync(slot, S.x[cur], sizeof(F) * n, cudaMemcpyDeviceToDevice, st))) return e;
    if ((e = cudaMemcpyAsync(slot + n, S.y[cur], sizeof(F) * m, cudaMemcpyDeviceToDevice, st))) return e;
    k_unr_segment<<<1, 64, 0, st>>>(S.s);
    const long long k_end = std::min<long long>(T, (long long)(sg + 1) * ckpt);
    for (;;) {
      e = pg.grid > 0 ? launch_persist<F>(K, KT, P, S2, pg, st) : launch_step_pair<F>(K, KT, P, S2, st);
      if (e) return e;
      if ((e = cudaMemcpyAsync(&h, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st))) return e;
      if ((e = cudaStreamSynchronize(st))) return e;
      if (h.err) {
        U.status = kWaitTimeout;
        return cudaSuccess;
      }
      if (h.status != kRunning) {
        U.status = h.status;
        return cudaSuccess;
      }
      if (h.k >= k_end) break;
      if (h.attempts >= in2.attempt_limit) {
        U.status = kKktLimit;
        return cudaSuccess;
      }
    }
    cur = h.cur;
  }
  U.omega = h.omega;
  U.inv_omega = h.inv_omega;
  k_unr_out<F><<<ew_grid(n + m), kEw, 0, st>>>(n, m, S.x[cur], S.y[cur], P.D2, P.D1, U.xo, U.yo);
  U.eta_host.resize((size_t)T);
  if ((e = cudaMemcpyAsync(U.eta_host.data(), U.eta, sizeof(double) * T, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  U.status = kOptimal;  // the map ran to T steps
  U.ready = true;
  return cudaGetLastError();
}

template <typename F>
cudaError_t unroll_backward(UnrollBuffers &U, const Mat<F> &Kf, const Mat<F> &KTf, const Problem<F> &Pf,
                            const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                            const double *dL_dx, const double *dL_dy, cudaStream_t st) {
  cudaError_t e;
  const int n = P.n, m = P.m, L = U.ckpt;
  const int64_t nnz = U.nnz;
  // segment store: xe, y_t (float64) and the two masks per step
  char *seg = reinterpret_cast<char *>(U.seg.get((sizeof(double) + 1) * (size_t)L * (n + m)));
  double *work = reinterpret_cast<double *>(U.work.get(sizeof(double) * (size_t)(6 * n + 8 * m)));
  F *fwork = reinterpret_cast<F *>(U.fwork.get(sizeof(F) * (size_t)(2 * n + 4 * m)));
  double *grads = reinterpret_cast<double *>(U.grads.get(sizeof(double) * (size_t)(2 * (n + m) + 2 * nnz)));
  const int32_t *row = U.row;
  if (!seg || !work || !fwork || !grads || !row) return cudaErrorMemoryAllocation;
  double *XE = reinterpret_cast<double *>(seg);
  double *YS = XE + (size_t)L * n;
  uint8_t *MX = reinterpret_cast<uint8_t *>(YS + (size_t)L * m);
  uint8_t *MY = MX + (size_t)L * n;
  double *w = work;
  double *xbar = w + 2 * n, *g = w + 3 * n, *gx = w + 4 * n;
  double *ybar = w + 6 * n + 4 * m, *h = ybar + m, *gy = ybar + 2 * m;
  F *xa = fwork, *xb2 = fwork + n, *ya = fwork + 2 * n, *yb2 = ya + m, *Kxa = ya + 2 * m, *Kxb = ya + 3 * m;
  double *dcs = grads, *dqs = grads + n, *dKs = grads + n + m;
  U.dc = dKs + nnz;
  U.dq = U.dc + n;
  U.dK = U.dq + m;
  if ((e = cudaMemcpyAsync(gx, dL_dx, sizeof(double) * n, cudaMemcpyDefault, st))) return e;
  if (dL_dy && (e = cudaMemcpyAsync(gy, dL_dy, sizeof(double) * m, cudaMemcpyDefault, st))) return e;
  k_adj_init<<<ew_grid(n + m), kEw, 0, st>>>(n, m, gx, dL_dy ? gy : nullptr, P.D2, P.D1, xbar, ybar);
  if ((e = cudaMemsetAsync(grads, 0, sizeof(double) * (size_t)(n + m + nnz), st))) return e;
  const size_t sm1 = spmv_bytes<double>(), smf = spmv_bytes<F>();
  const F *ck = reinterpret_cast<const F *>(U.ckpts.ptr());
  for (int sg = U.nseg - 1; sg >= 0; --sg) {
    const int t0 = sg * L, len = std::min(L, U.T - t0);
    if ((e = cudaMemcpyAsync(xa, ck + (size_t)sg * (n + m), sizeof(F) * n, cudaMemcpyDeviceToDevice, st)))
      return e;
    if ((e = cudaMemcpyAsync(ya, ck + (size_t)sg * (n + m) + n, sizeof(F) * m, cudaMemcpyDeviceToDevice, st)))
      return e;
    launch_spmv<F>(Kf, xa, Kxa, st);
    F *xc = xa, *xn = xb2, *yc = ya, *yn = yb2, *kc = Kxa, *kn = Kxb;
    for (int t = 0; t < len; ++t) {
      // the forward arithmetic: tau, sigma as the step kernels form them
      const double eta = U.eta_host[(size_t)(t0 + t)];
      const F tau = (F)(eta * U.inv_omega), sigma = (F)(eta * U.omega);
      if (KTf.nblocks > 0)
        k_unr_primal<F><<<KTf.nblocks, kThreads, smf, st>>>(KTf, Pf, xc, yc, xn, XE + (size_t)t * n,
                                                            MX + (size_t)t * n, tau);
      k_unr_dual<F><<<Kf.nblocks, kThreads, smf, st>>>(Kf, Pf, xn, kc, yc, yn, kn, YS + (size_t)t * m,
                                                       MY + (size_t)t * m, sigma);
      std::swap(xc, xn);
      std::swap(yc, yn);
      std::swap(kc, kn);
    }
    for (int t = len - 1; t >= 0; --t) {
      // the adjoint in float64 with the float64 K~ (the step sizes of the map)
      const double eta = U.eta_host[(size_t)(t0 + t)];
      const double tau = (double)(F)(eta * U.inv_omega), sigma = (double)(F)(eta * U.omega);
      k_adj_h<<<ew_grid(m), kEw, 0, st>>>(m, ybar, MY + (size_t)t * m, h);
      if (KT.nblocks > 0)
        k_adj_cols<<<KT.nblocks, kThreads, sm1, st>>>(KT, h, MX + (size_t)t * n, xbar, g, dcs, tau, sigma);
      k_adj_rows<<<K.nblocks, kThreads, sm1, st>>>(K, g, h, ybar, dqs, tau, sigma);
      k_adj_dK<<<ew_grid(nnz), kEw, 0, st>>>(nnz, row, K.ci, h, YS + (size_t)t * m, XE + (size_t)t * n, g, dKs, tau,
                                             sigma);
    }
    if ((e = cudaGetLastError())) return e;
  }
  k_adj_final<<<ew_grid(n + m), kEw, 0, st>>>(n, m, P.D2, P.D1, dcs, dqs, U.dc, U.dq);
  k_adj_final_K<<<ew_grid(nnz), kEw, 0, st>>>(nnz, row, K.ci, P.D1, P.D2, dKs, U.dK);
  return cudaGetLastError();
}

#define PDLP_INST(F)                                                                                          \
  template cudaError_t unroll_forward<F>(UnrollBuffers &, const Mat<F> &, const Mat<F> &, const Problem<F> &,  \
                                         const State<F> &, const PersistGeo &, const ScalarInit &, double,       \
                                         double *, int32_t, int32_t, const double *, const double *,              \
                                         cudaStream_t);                                                            \
  template cudaError_t unroll_backward<F>(UnrollBuffers &, const Mat<F> &, const Mat<F> &, const Problem<F> &, \
                                          const Mat<double> &, const Mat<double> &, const Problem<double> &,      \
                                          const double *, const double *, cudaStream_t);
PDLP_INST(double)
PDLP_INST(float)
#undef PDLP_INST

}  // namespace pdlp
