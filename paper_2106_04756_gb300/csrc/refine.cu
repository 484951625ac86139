// Iterative refinement: float32 PDLP solves of correction problems inside a
// float64 outer loop.
//
// At a point (xh, yh) of the original LP, with primal violation pv (largest
// |q - K xh| on equality rows, (q - K xh)^+ on inequality rows, bound
// violations) and dual violation dv (largest |c - K^T yh - lambda| with
// lambda = proj_Lambda(c - K^T yh), and dual sign violations), the correction
// problem is the saddle problem of Eq. (2) with the same K and
//     c' = dD (c - K^T yh),  q' = dP (q - K xh),
//     l' = dP (l - xh),      u' = dP (u - xh),  y_i >= -dD (yh_i - ylo_i) on inequality rows,
// dP = 1/pv, dD = 1/dv (clipped to [1, dmax]).  Scaling the Lagrangian by the
// positive factor dP dD maps its saddle points (a, b) one to one onto those
// of the original problem: x = xh + a/dP, y = yh + b/dD.  Each round solves
// the correction problem in float32 to a loose tolerance and applies the
// correction in float64; the loop stops when Eq. (15) holds on the original
// problem, evaluated in float64.  When a round divides the error by less than
// kRefineMinGain (the float32 solves of the corrections have stalled), makes
// it worse, or the round cap is reached, the loop hands the best point to a
// float64 PDLP finish (run by the caller) with what is left of the budget:
// every inner solve and the finish share the caller's iteration, KKT-pass
// and time limits.
#include <math.h>

#include <chrono>
#include <vector>

#include "refine.cuh"
#include "solver.cuh"

namespace pdlp {

namespace {

__device__ __forceinline__ double proj_lam(double rc, double l, double u) {
  const bool lf = l > -INFINITY, uf = u < INFINITY;
  if (!lf && !uf) return 0.0;
  if (!lf) return rc < 0.0 ? rc : 0.0;
  if (!uf) return rc > 0.0 ? rc : 0.0;
  return rc;
}

// scaled copies of the current point: x~ = xh / D2, y~ = yh / D1
__global__ void k_ref_scale(int32_t n, int32_t m, const double *xh, const double *yh, const double *D1,
                            const double *D2, double *xt, double *yt) {
  const int N = n + m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) xt[i] = xh[i] / D2[i];
    else yt[i - n] = yh[i - n] / D1[i - n];
  }
}

// Column and row terms of Eq. (15) at (xh, yh) and the violations.
// partc per CTA: pobj, dres^2, dobj(lambda), max dual violation, max primal (bound) violation
// partr per CTA: pres^2, dobj(q), max primal violation, max dual sign violation
__global__ void k_ref_eval(Problem<double> P, RefView R) {
  __shared__ double red[5 * 8];
  __shared__ double mred[3 * 8];
  double acc[5] = {0, 0, 0, 0, 0};
  double pvmax = 0.0, dvmax = 0.0, bvmax = 0.0;
  const int n = P.n, N = P.n + P.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double x = R.xh[i], c = P.c[i], l = P.l[i], u = P.u[i];
      const double rc = c - R.KTy[i] / P.D2[i];
      const double lam = proj_lam(rc, l, u);
      acc[0] += c * x;
      acc[1] += (rc - lam) * (rc - lam);
      acc[2] += (lam > 0.0 ? l * lam : 0.0) + (lam < 0.0 ? u * lam : 0.0);
      dvmax = fmax(dvmax, fabs(rc - lam));
      bvmax = fmax(bvmax, fmax(l - x, x - u));
    } else {
      const int r = i - n;
      const double lo = P.ylo[r], y = R.yh[r], q = P.q[r];
      double res = q - R.Kx[r] / P.D1[r];
      double viol = fabs(res);
      if (lo > -INFINITY) {
        if (lo != 0.0) acc[0] += lo * res;
        res = res > 0.0 ? res : 0.0;
        viol = res;
        dvmax = fmax(dvmax, lo - y);
      }
      acc[3] += res * res;
      acc[4] += q * y;
      pvmax = fmax(pvmax, viol);
    }
  }
  block_sum<5>(acc, red);
  // maxima: warp then CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    pvmax = fmax(pvmax, __shfl_down_sync(0xffffffffu, pvmax, o));
    dvmax = fmax(dvmax, __shfl_down_sync(0xffffffffu, dvmax, o));
    bvmax = fmax(bvmax, __shfl_down_sync(0xffffffffu, bvmax, o));
  }
  __syncthreads();
  if (lane == 0) { mred[warp] = pvmax; mred[8 + warp] = dvmax; mred[16 + warp] = bvmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      pvmax = fmax(pvmax, mred[w]);
      dvmax = fmax(dvmax, mred[8 + w]);
      bvmax = fmax(bvmax, mred[16 + w]);
    }
    double *p = R.partc + 8 * blockIdx.x;
    for (int a = 0; a < 5; ++a) p[a] = acc[a];
    p[5] = fmax(pvmax, bvmax);
    p[6] = dvmax;
  }
  if (!last_block(R.ticket)) return;
  double tot[5];
  sum_partials<5>(R.partc, gridDim.x, 8, tot, red);
  if (threadIdx.x == 0) {
    double pv = 0.0, dv = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      pv = fmax(pv, __ldcg(R.partc + 8 * b + 5));
      dv = fmax(dv, __ldcg(R.partc + 8 * b + 6));
    }
    const double pobj = tot[0], dobj = tot[2] + tot[4];
    const double pres = sqrt(tot[3]), dres = sqrt(tot[1]), gap = fabs(dobj - pobj);
    double *k = R.rsc;
    k[0] = pobj;
    k[1] = dobj;
    k[2] = gap;
    k[3] = pres;
    k[4] = dres;
    k[8] = pv;
    k[9] = dv;
  }
}

// Builds the correction problem at (xh, yh) with scales dP, dD.
__global__ void k_ref_build(Problem<double> P, RefView R, double dP, double dD) {
  const int n = P.n, N = P.n + P.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double D2 = P.D2[i], x = R.xh[i];
      const double c = dD * (P.c[i] - R.KTy[i] / D2);
      const double l = dP * (P.l[i] - x), u = dP * (P.u[i] - x);
      R.c[i] = c;
      R.l[i] = l;
      R.u[i] = u;
      R.cs[i] = (float)(D2 * c);
      R.ls[i] = (float)(l / D2);
      R.us[i] = (float)(u / D2);
    } else {
      const int r = i - n;
      const double D1 = P.D1[r], lo = P.ylo[r];
      const double q = dP * (P.q[r] - R.Kx[r] / D1);
      const double yl = lo > -INFINITY ? -dD * (R.yh[r] - lo) : -INFINITY;
      R.q[r] = q;
      R.ylo[r] = yl;
      R.qs[r] = (float)(D1 * q);
      R.ylos[r] = (float)(yl / D1);
    }
  }
}

// xh += a / dP, yh += b / dD, projected onto X x Y.
__global__ void k_ref_update(Problem<double> P, RefView R, const double *a, const double *b, double dP,
                             double dD) {
  const int n = P.n, N = P.n + P.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double x = R.xh[i] + a[i] / dP;
      R.xh[i] = fmin(fmax(x, P.l[i]), P.u[i]);
    } else {
      const int r = i - n;
      const double y = R.yh[r] + b[r] / dD;
      R.yh[r] = fmax(y, P.ylo[r]);
    }
  }
}

__global__ void k_ref_start(Problem<double> P, RefView R, const double *x0, const double *y0) {
  const int n = P.n, N = P.n + P.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (i < n) R.xh[i] = fmin(fmax(x0[i], P.l[i]), P.u[i]);
    else R.yh[i - n] = fmax(y0[i - n], P.ylo[i - n]);
  }
}

}  // namespace

cudaError_t refine_alloc(RefineBuffers &R, int32_t m, int32_t n, int32_t nbK, int32_t nbKT) {
  if (R.ready) return cudaSuccess;
  R.m = m;
  R.n = n;
  R.nbK = nbK;
  R.nbKT = nbKT;
  const size_t nd = 5 * (size_t)n + 5 * (size_t)m + 3 * (size_t)n + 2 * (size_t)m;
  double *d = reinterpret_cast<double *>(R.vec.get(sizeof(double) * nd));
  float *f = reinterpret_cast<float *>(R.vec32.get(sizeof(float) * (3 * (size_t)n + 2 * (size_t)m)));
  double *part = reinterpret_cast<double *>(R.part.get(sizeof(double) * 8 * 1024 + 64));
  double *rs = reinterpret_cast<double *>(R.rs.get(sizeof(double) * 16));
  double *tl = reinterpret_cast<double *>(R.tol.get(sizeof(double)));
  if (!d || !f || !part || !rs || !tl) return cudaErrorMemoryAllocation;
  R.v.xh = d; d += n;
  R.v.yh = d; d += m;
  R.v.xt = d; d += n;
  R.v.yt = d; d += m;
  R.v.Kx = d; d += m;
  R.v.KTy = d; d += n;
  R.v.xb = d; d += n;
  R.v.yb = d; d += m;
  R.v.c = d; d += n;
  R.v.q = d; d += m;
  R.v.l = d; d += n;
  R.v.u = d; d += n;
  R.v.ylo = d; d += m;
  R.v.cs = f; f += n;
  R.v.ls = f; f += n;
  R.v.us = f; f += n;
  R.v.qs = f; f += m;
  R.v.ylos = f; f += m;
  R.v.partc = part;
  R.v.ticket = reinterpret_cast<unsigned *>(part + 8 * 1024);
  R.v.rsc = rs;
  cudaError_t e = cudaMemset(R.v.ticket, 0, 64);
  if (e) return e;
  e = cudaMemset(R.vec32.ptr(), 0, sizeof(float) * (3 * (size_t)n + 2 * (size_t)m));
  if (e) return e;
  e = cudaMemset(R.vec.ptr(), 0, sizeof(double) * nd);
  if (e) return e;
  R.ready = true;
  return cudaSuccess;
}

long long *refine_limits_dev(RefineBuffers &R) {
  return reinterpret_cast<long long *>(R.lim.get(4 * sizeof(long long)));
}

int refine_set_limits(RefineBuffers &R, const RefineLimits &L, long long iters, long long passes, double secs,
                      cudaStream_t st, int *spent, cudaError_t *err) {
  long long left[3];
  const int why = refine_remaining(L.iter_limit, L.kkt_limit, L.time_limit_s, iters, passes, secs, left);
  *err = cudaSuccess;
  if (why) {
    *spent = why == 1 ? kIterLimit : (why == 2 ? kKktLimit : kTimeLimit);
    return 0;
  }
  long long *d = refine_limits_dev(R);
  if (!d) {
    *err = cudaErrorMemoryAllocation;
    return 0;
  }
  // pageable source: the copy is staged before the call returns
  *err = cudaMemcpyAsync(d, left, sizeof(left), cudaMemcpyHostToDevice, st);
  return *err == cudaSuccess ? 1 : 0;
}

Problem<float> refine_problem(RefineBuffers &R, const Problem<double> &P64) {
  Problem<float> P;
  P.m = P64.m;
  P.n = P64.n;
  P.cs = R.v.cs;
  P.qs = R.v.qs;
  P.ls = R.v.ls;
  P.us = R.v.us;
  P.ylos = R.v.ylos;
  P.c = R.v.c;
  P.q = R.v.q;
  P.l = R.v.l;
  P.u = R.v.u;
  P.ylo = R.v.ylo;
  P.D1 = P64.D1;
  P.D2 = P64.D2;
  P.D1inv = P64.D1inv;
  P.D2inv = P64.D2inv;
  return P;
}

cudaError_t refine_solve(RefineBuffers &R, const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                         const State<float> &Sc, const std::function<cudaError_t(Scalars *)> &run_inner,
                         double tol, double inner_tol, int max_rounds, const RefineLimits &lim,
                         const double *x_stage, const double *y_stage, cudaStream_t st, RefineOutcome *out) {
  cudaError_t e;
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(); };
  const int N = P.n + P.m, grid = (N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024;
  RefView V = R.v;
  k_ref_start<<<grid, 256, 0, st>>>(P, V, x_stage, y_stage);
  // ||q||, ||c|| of the original problem for the relative terms of Eq. (15)
  std::vector<double> hq(P.m), hc(P.n);
  if ((e = cudaMemcpyAsync(hq.data(), P.q, sizeof(double) * P.m, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(hc.data(), P.c, sizeof(double) * P.n, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  double qn = 0.0, cn = 0.0;
  for (double v : hq) qn += v * v;
  for (double v : hc) cn += v * v;
  qn = sqrt(qn);
  cn = sqrt(cn);
  const int egrid = 256 < grid ? 256 : grid;
  double h[16];
  Scalars hs;
  out->status = kIterLimit;
  out->iters = out->kkt_passes = out->restarts = 0;
  out->rounds = 0;
  out->finish = false;
  double best = INFINITY;
  int inner_stop = 0;  // an inner solve stopped at a limit: end after evaluating its update
  for (int round = 0;; ++round) {
    k_ref_scale<<<grid, 256, 0, st>>>(P.n, P.m, V.xh, V.yh, P.D1, P.D2, V.xt, V.yt);
    launch_spmv<double>(K, V.xt, V.Kx, st);
    launch_spmv<double>(KT, V.yt, V.KTy, st);
    k_ref_eval<<<egrid, 256, 0, st>>>(P, V);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemcpyAsync(h, V.rsc, sizeof(double) * 16, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    h[5] = h[2] / (1.0 + fabs(h[1]) + fabs(h[0]));
    h[6] = h[3] / (1.0 + qn);
    h[7] = h[4] / (1.0 + cn);
    const double rel = fmax(h[5], fmax(h[6], h[7]));
    if (!(rel < best)) {
      // the last correction did not improve Eq. (15): keep the best point
      if ((e = cudaMemcpyAsync(V.xh, V.xb, sizeof(double) * P.n, cudaMemcpyDeviceToDevice, st))) return e;
      if ((e = cudaMemcpyAsync(V.yh, V.yb, sizeof(double) * P.m, cudaMemcpyDeviceToDevice, st))) return e;
      if ((e = cudaStreamSynchronize(st))) return e;
      if (inner_stop) out->status = inner_stop;
      else out->finish = isfinite(best);
      break;
    }
    const double prev = best;
    best = rel;
    for (int a = 0; a < 8; ++a) out->kkt[a] = h[a];
    out->rounds = round;
    if (h[5] <= tol && h[6] <= tol && h[7] <= tol) { out->status = kOptimal; break; }
    if (!(isfinite(h[0]) && isfinite(h[1]))) { out->status = kNumErr; break; }
    if (inner_stop) { out->status = inner_stop; break; }
    if (refine_finish_now(round, prev, rel, max_rounds)) { out->finish = true; break; }
    int spent = 0;
    if (!refine_set_limits(R, lim, out->iters, out->kkt_passes, elapsed(), st, &spent, &e)) {
      if (e) return e;
      out->status = spent;
      break;
    }
    if ((e = cudaMemcpyAsync(V.xb, V.xh, sizeof(double) * P.n, cudaMemcpyDeviceToDevice, st))) return e;
    if ((e = cudaMemcpyAsync(V.yb, V.yh, sizeof(double) * P.m, cudaMemcpyDeviceToDevice, st))) return e;
    double dP, dD;
    refine_scales(h[8], h[9], 1e12, &dP, &dD);
    k_ref_build<<<grid, 256, 0, st>>>(P, V, dP, dD);
    // inner float32 solve from zero (the staging buffers are the graph's start point)
    const double round_tol = refine_round_tol(rel, tol, inner_tol);
    if ((e = cudaMemcpyAsync(R.tol.ptr(), &round_tol, sizeof(double), cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemsetAsync(const_cast<double *>(x_stage), 0, sizeof(double) * P.n, st))) return e;
    if ((e = cudaMemsetAsync(const_cast<double *>(y_stage), 0, sizeof(double) * P.m, st))) return e;
    if ((e = run_inner(&hs))) return e;
    k_ref_update<<<grid, 256, 0, st>>>(P, V, Sc.xo, Sc.yo, dP, dD);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    out->iters += hs.k;
    out->kkt_passes += hs.attempts;
    out->restarts += hs.restarts;
    if (hs.status == kTimeLimit || hs.status == kIterLimit || hs.status == kKktLimit) inner_stop = hs.status;
  }
  out->x = V.xh;
  out->y = V.yh;
  out->seconds = elapsed();
  return cudaSuccess;
}

}  // namespace pdlp
