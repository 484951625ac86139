// Batched solve of many small LPs in one persistent launch (pdlp_solve_batch).
//
// One CTA runs the whole method on one LP at a time and takes the next LP
// from a queue ordered largest first: the transpose of K (counting sort by
// column, then each column ordered by row), Ruiz (10 passes) and
// Pock-Chambolle (alpha = 1) scaling (Section 3.5), the data transform, the
// initialisation of Algorithm 1, step attempts of Algorithm 2, the running
// average, and every eval_every steps the Eq. (15) test on the original
// problem, the restart candidate and criteria of Section 3.2 with the
// normalized duality gap, and the primal weight of Algorithm 3.  The
// arithmetic of each step is that of the single-LP path; reductions are
// fixed-order CTA sums in float64.  The products use L lanes per row (L a
// power of two chosen per LP by the autotuner); the normalized gap sorts the
// breakpoints of the trust-region problem in shared memory (bitonic) and
// locates the crossing segment with prefix sums.
//
// Per-CTA workspace (global memory, sized for the largest LP of the batch)
// holds the scaled problem, K^T and the iterates; with one LP per SM at a time
// the working set of the resident CTAs stays in L2.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "prep.cuh"

namespace pdlp {
void set_last_error(const std::string &msg);
}

namespace pdlp {
namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kSortMax = 4096;  // n + m of one LP (breakpoint sort in shared memory)
constexpr int kNumBuckets = 5;  // by mean row length of K: <8, <16, <32, <64, >=64
// dynamic shared memory: the breakpoint sort, or the product tile of a product
constexpr size_t kBatchSmem = 96 * 1024;
static_assert(kBatchSmem >= (size_t)kSortMax * (sizeof(double) + sizeof(int)), "sort buffer");

struct BatchIn {
  int32_t count;
  const int32_t *m, *n;
  const int64_t *row_off, *col_off, *nnz_off;
  const int32_t *rp, *ci;
  const double *val, *c, *q, *l, *u;
  const uint8_t *ineq;
  const int32_t *order;  // LP processing order
  const int32_t *lanes;  // per LP: lanes per row for K (low byte) and K^T (next byte)
  // nullable: starting points (original space, packed like c / q) and the
  // iterations / KKT passes each LP already spent (its limits shrink by them)
  const double *x0, *y0;
  const long long *used_iters, *used_passes;
};

struct BatchOpts {
  double rel_tol, eps_zero, beta_suff, beta_nec, beta_art, pw_theta, primal_importance;
  long long iter_limit, kkt_pass_limit;
  int ruiz_iters, pock_chambolle, eval_every, adaptive_restart, pw_update;
  int restart_to_current;  // 0: the restart candidate is always the average (Appendix C.2)
  int stall_evals;         // > 0: stop (kStalled) after this many evaluations without a 10% gain
};

struct BatchOut {
  double *x, *y;        // original space, packed like c / q
  pdlp_result *res;     // per LP (device)
  unsigned *queue;      // next LP to take
  unsigned *bad;        // first invalid LP + 1 (0: none)
};

// Workspace of one CTA, carved from a slab sized for (mm, nn, zz).
template <typename T>
struct Work {
  double *D1, *D2, *kv, *ktv, *cs, *qs, *ls, *us, *ylos, *tmpm, *tmpn;
  int32_t *trp, *tci, *perm, *fill, *rpk;
  T *k, *kt;  // K~ and K~^T values in the arithmetic type
  T *x[2], *y[2], *Kx[2], *x0, *y0, *xa, *ya;
  double *xs[2], *ys[2];  // running sums of the average, float64 whatever T
  T *csT, *lsT, *usT, *qsT, *yloT;  // scaled data in the arithmetic type
  double *gt, *ga, *gw, *gv;  // gap items
  // products of the evaluation (Eq. (15), normalized gap), float64 whatever
  // T: K^T y and K x of the current iterate, of the average
  double *KTyd, *Kxd, *KTysd, *Kxsd;
};

template <typename T>
size_t work_bytes(int mm, int nn, long long zz) {
  const size_t d = sizeof(double) * (size_t)(4 * zz + 10 * (size_t)nn + 8 * (size_t)mm + 4 * (size_t)(nn + mm));
  const size_t i = sizeof(int32_t) * (size_t)(2 * zz + 2 * (size_t)nn + (size_t)mm + 3);
  const size_t t = sizeof(T) * (size_t)(2 * zz + 12 * (size_t)nn + 11 * (size_t)mm) + 64;
  return (d + i + t + 255) / 256 * 256;
}

template <typename T>
__device__ Work<T> carve(char *base, int mm, int nn, long long zz) {
  Work<T> w;
  double *d = reinterpret_cast<double *>(base);
  auto tk = [&](size_t k) { double *r = d; d += k; return r; };
  w.D1 = tk(mm); w.D2 = tk(nn); w.kv = tk(zz); w.ktv = tk(zz);
  w.cs = tk(nn); w.qs = tk(mm); w.ls = tk(nn); w.us = tk(nn); w.ylos = tk(mm);
  w.tmpm = tk(mm); w.tmpn = tk(nn);
  w.gt = tk(nn + mm); w.ga = tk(nn + mm); w.gw = tk(nn + mm); w.gv = tk(nn + mm);
  tk(2 * zz);  // spare (keeps the formula simple)
  w.KTyd = tk(nn); w.KTysd = tk(nn); w.Kxd = tk(mm); w.Kxsd = tk(mm);
  w.xs[0] = tk(nn); w.xs[1] = tk(nn); w.ys[0] = tk(mm); w.ys[1] = tk(mm);
  int32_t *ip = reinterpret_cast<int32_t *>(d);
  w.trp = ip; ip += nn + 1;
  w.tci = ip; ip += zz;
  w.perm = ip; ip += zz;
  w.fill = ip; ip += nn + 1;
  w.rpk = ip; ip += mm + 1;
  T *t = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(ip) + 15) & ~uintptr_t(15));
  auto tt = [&](size_t k) { T *r = t; t += k; return r; };
  w.k = tt(zz); w.kt = tt(zz);
  w.x[0] = tt(nn); w.x[1] = tt(nn); w.x0 = tt(nn);
  w.xa = tt(nn);
  w.y[0] = tt(mm); w.y[1] = tt(mm); w.Kx[0] = tt(mm); w.Kx[1] = tt(mm);
  w.y0 = tt(mm); w.ya = tt(mm);
  w.csT = tt(nn); w.lsT = tt(nn); w.usT = tt(nn); w.qsT = tt(mm); w.yloT = tt(mm);
  return w;
}

// ------------------------------------------------------------ CTA helpers

// Fixed-order CTA sum of NV values; the result is returned in every thread
// (thread 0 adds the warp partials; float64 is slow on this part, so the
// final adds are not repeated in every thread).
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * kBWarps + warp] = v[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = 0.0;
      for (int w = 0; w < kBWarps; ++w) t += red[a * kBWarps + w];
      red[NV * kBWarps + a] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = red[NV * kBWarps + a];
  __syncthreads();
}

// The same sum for NV <= 3 with few float64 adds (float64 is slow on this
// part): values to shared memory, warp 0 adds kBThreads / 32 per lane, then a
// 5-step shuffle; the result is returned in every thread.
template <int NV>
__device__ __forceinline__ void cta_sum_lean(double (&v)[NV], double *red) {
  static_assert(NV <= 3, "red holds 3 x kBThreads doubles");
  const int lane = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) red[a * kBThreads + threadIdx.x] = v[a];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = 0.0;
      for (int k = lane; k < kBThreads; k += 32) t += red[a * kBThreads + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[a] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[3 * kBThreads + a] = v[a];
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = red[3 * kBThreads + a];
}

__device__ __forceinline__ double cta_max(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = red[0];
  for (int w = 1; w < kBWarps; ++w) t = fmax(t, red[w]);
  __syncthreads();
  return t;
}

// Row sums of a CSR block (rows, rp with rows + 1 entries, values a, columns
// ci) with L lanes per row; epi(row, sum) runs in the row's first lane.
// Two passes per tile of whole rows with at most `cap` nonzeros: every
// product a_k v[ci_k] of the tile is formed with all its loads independent
// (coalesced a and ci, gathered v) into shared memory `prod`, then each row
// is summed from shared memory (fixed order: lane gl takes k = s + gl,
// s + gl + L, ..., then a shuffle tree).  A row longer than `cap` is summed
// directly from global memory.
template <typename T, typename TV = T, typename Epi>
__device__ __forceinline__ void cta_spmv(int rows, const int32_t *rp, const int32_t *ci, const T *a, const TV *v,
                                         int L, T *prod, int cap, Epi &&epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = 32 / L, g = lane / L, gl = lane % L;
  int r0 = 0;
  while (r0 < rows) {
    // last row end r1 with rp[r1] - rp[r0] <= cap (same in every thread)
    const int base = rp[r0];
    int lo = r0, hi = rows;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rp[mid] - base <= cap) lo = mid;
      else hi = mid - 1;
    }
    int r1 = lo;
    if (r1 == r0) {  // one row longer than the tile: direct sum by warp 0
      if (warp == 0) {
        T acc = T(0);
        for (int k = base + lane; k < rp[r0 + 1]; k += 32) acc = fma(a[k], (T)v[ci[k]], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) epi(r0, acc);
      }
      __syncthreads();
      r0 += 1;
      continue;
    }
    const int cnt = rp[r1] - base;
    for (int e0 = threadIdx.x; e0 < cnt; e0 += 4 * kBThreads) {
      T av[4], vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * kBThreads;
        av[u] = e < cnt ? a[base + e] : T(0);
        vv[u] = e < cnt ? (T)v[ci[base + e]] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * kBThreads;
        if (e < cnt) prod[e] = av[u] * vv[u];
      }
    }
    __syncthreads();
    for (int rb = r0 + warp * per; rb < r1; rb += kBWarps * per) {
      const int r = rb + g;
      T acc = T(0);
      if (r < r1) {
        const int e = rp[r + 1] - base;
        for (int k = rp[r] - base + gl; k < e; k += L) acc += prod[k];
      }
      for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, L);
      if (r < r1 && gl == 0) epi(r, acc);
    }
    __syncthreads();
    r0 = r1;
  }
}

__device__ __forceinline__ double lam_of(double rc, double l, double u) {
  const bool lf = l > -INFINITY, uf = u < INFINITY;
  if (!lf && !uf) return 0.0;
  if (!lf) return rc < 0.0 ? rc : 0.0;
  if (!uf) return rc > 0.0 ? rc : 0.0;
  return rc;
}

// Section 3.2 normalized gap at z = (x, y) with gradient (KTy - c, q - Kx),
// weight om and radius r: items into global scratch, (t, index) sorted in
// shared memory, then the first breakpoint whose phi reaches r^2 by prefix
// sums.  Returns +inf for r = 0.
template <typename T>
__device__ double cta_gap(const Work<T> &w, int n, int m, const T *x, const T *y, const double *KTy,
                          const double *Kx, double om, double r, double *skey, int *sidx, double *red) {
  if (!(r > 0.0)) return INFINITY;
  const int N = n + m;
  int P = 1;
  while (P < N) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    double t = INFINITY, a = 0.0, wv = 0.0, vv = 0.0;
    bool item = false;
    if (i < n) {
      const double g = (double)KTy[i] - w.cs[i];
      if (g != 0.0) {
        item = true;
        double dist = g > 0.0 ? w.us[i] - (double)x[i] : (double)x[i] - w.ls[i];
        if (!(dist > 0.0)) dist = 0.0;
        const double ag = fabs(g);
        a = g * g / om;
        if (!isinf(dist)) {
          t = om * dist / ag;
          wv = om * dist * dist;
          vv = ag * dist;
        }
      }
    } else if (i < N) {
      const int k = i - n;
      const double g = w.qs[k] - (double)Kx[k];
      if (g != 0.0) {
        item = true;
        double dist = g > 0.0 ? INFINITY : (double)y[k] - w.ylos[k];
        if (!(dist > 0.0)) dist = 0.0;
        const double ag = fabs(g);
        a = om * g * g;
        if (!isinf(dist)) {
          t = dist / (om * ag);
          wv = dist * dist / om;
          vv = ag * dist;
        }
      }
    }
    if (i < N) {
      w.gt[i] = t;
      w.ga[i] = item ? a : 0.0;
      w.gw[i] = wv;
      w.gv[i] = vv;
    }
    skey[i] = i < N ? t : INFINITY;
    sidx[i] = i;
  }
  __syncthreads();
  // bitonic sort of (key, index) ascending
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          const double a = skey[i], b = skey[p];
          const int ia = sidx[i], ib = sidx[p];
          const bool gt = a > b || (a == b && ia > ib);
          if (gt == up) {
            skey[i] = b;
            skey[p] = a;
            sidx[i] = ib;
            sidx[p] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  // per thread a contiguous run of the sorted items: prefix of w and v,
  // suffix of a; then the first k with W_k + t_k^2 A_k >= r^2
  const int per = (P + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(b0 + per, P);
  double sw = 0.0, sv = 0.0, sa = 0.0;
  for (int i = b0; i < b1; ++i) {
    const int id = sidx[i];
    if (id < N) {
      sw += w.gw[id];
      sv += w.gv[id];
      sa += w.ga[id];
    }
  }
  // exclusive scans (fixed order) over the thread runs
  double *pw = red, *pv = red + blockDim.x, *pa = red + 2 * blockDim.x;
  pw[threadIdx.x] = sw;
  pv[threadIdx.x] = sv;
  pa[threadIdx.x] = sa;
  __syncthreads();
  if (threadIdx.x == 0) {
    double aw = 0.0, av = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const double a0 = pw[t], a1 = pv[t];
      pw[t] = aw;
      pv[t] = av;
      aw += a0;
      av += a1;
    }
    double as = 0.0;
    for (int t = (int)blockDim.x - 1; t >= 0; --t) {
      as += pa[t];
      pa[t] = as;  // inclusive suffix from t
    }
  }
  __syncthreads();
  const double target = r * r;
  double W = pw[threadIdx.x], V = pv[threadIdx.x];
  double A = pa[threadIdx.x];  // sum of a over runs t.. (this run included)
  int found = P;
  double fW = 0.0, fV = 0.0, fA = 0.0;
  for (int i = b0; i < b1; ++i) {
    const int id = sidx[i];
    const double t = skey[i];
    const bool real = id < N;
    if (!(t < INFINITY)) {  // first infinite breakpoint: stop here
      found = i;
      fW = W;
      fV = V;
      fA = A;
      break;
    }
    const double phi = W + t * t * A;
    if (phi >= target) {
      found = i;
      fW = W;
      fV = V;
      fA = A;
      break;
    }
    if (real) {
      W += w.gw[id];
      V += w.gv[id];
      A -= w.ga[id];
    }
  }
  // the smallest index that stopped wins
  int *sfound = reinterpret_cast<int *>(red + 3 * blockDim.x);
  if (threadIdx.x == 0) *sfound = P;
  __syncthreads();
  if (found < P) atomicMin(sfound, found);
  __syncthreads();
  const int kstar = *sfound;
  double *res = red + 3 * blockDim.x + 2;
  if (kstar == P) {
    if (threadIdx.x == blockDim.x - 1) {
      res[0] = W;
      res[1] = V;
      res[2] = 0.0;
    }
  } else if (kstar >= b0 && kstar < b1) {
    res[0] = fW;
    res[1] = fV;
    res[2] = fA;
  }
  __syncthreads();
  const double Wf = res[0], Vf = res[1], Af = res[2];
  __syncthreads();
  const double best = Af > 0.0 ? Vf + sqrt((target - Wf) / Af) * Af : Vf;
  return best / r;
}

template <typename T>
__global__ void __launch_bounds__(kBThreads) k_batch(BatchIn in, BatchOpts o, BatchOut out, char *slab,
                                                     size_t slab_bytes, int mm, int nn, long long zz) {
  extern __shared__ __align__(16) char bsm[];
  __shared__ double red[3 * kBThreads + 8];
  __shared__ double fac[2][kMaxEval];  // Algorithm 2 factors of the next eval_every steps
  __shared__ double s_step[4];
  __shared__ int s_lp;
  double *skey = reinterpret_cast<double *>(bsm);
  int *sidx = reinterpret_cast<int *>(skey + kSortMax);
  T *prod = reinterpret_cast<T *>(bsm);  // products of the current tile (not live with the sort)
  const int cap = (int)(kBatchSmem / sizeof(T));
  Work<T> w = carve<T>(slab + slab_bytes * blockIdx.x, mm, nn, zz);
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned j = atomicAdd(out.queue, 1u);
      s_lp = j < (unsigned)in.count ? in.order[j] : -1;
    }
    __syncthreads();
    const int b = s_lp;
    __syncthreads();
    if (b < 0) break;
    const int m = in.m[b], n = in.n[b];
    const int64_t ro = in.row_off[b], co = in.col_off[b], zo = in.nnz_off[b];
    const int nnz = (int)(in.nnz_off[b + 1] - zo);
    const int32_t *rp_in = in.rp + ro;  // m local offsets; row m ends at nnz
    const int32_t *ci = in.ci + zo;
    const double *val = in.val + zo, *c = in.c + co, *q = in.q + ro, *l = in.l + co, *u = in.u + co;
    const uint8_t *ineq = in.ineq + ro;
    const int Lk = in.lanes[b] & 0xff, Lt = (in.lanes[b] >> 8) & 0xff;
    const long long iter_limit = o.iter_limit - (in.used_iters ? in.used_iters[b] : 0ll);
    const long long pass_limit = o.kkt_pass_limit - (in.used_passes ? in.used_passes[b] : 0ll);
    // ---- validation (column range and order, finite data, l <= u)
    {
      int badl = 0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int s = rp_in[i], e = i + 1 < m ? rp_in[i + 1] : nnz;
        if (s < 0 || e < s || e > nnz) badl = 1;
        for (int k = s; k < e && !badl; ++k) {
          if (ci[k] < 0 || ci[k] >= n || (k > s && ci[k] <= ci[k - 1]) || !isfinite(val[k])) badl = 1;
        }
        if (!isfinite(q[i])) badl = 1;
      }
      for (int j = threadIdx.x; j < n; j += blockDim.x)
        if (!isfinite(c[j]) || !(l[j] <= u[j]) || l[j] == INFINITY || u[j] == -INFINITY) badl = 1;
      if (__syncthreads_or(badl)) {
        if (threadIdx.x == 0) atomicCAS(out.bad, 0u, (unsigned)b + 1u);
        continue;
      }
    }
    auto rbeg = [&](int i) { return rp_in[i]; };
    auto rend = [&](int i) { return i + 1 < m ? rp_in[i + 1] : nnz; };
    // ---- K^T: counts, scan, scatter, per-column order by row (a1)
    for (int j = threadIdx.x; j <= n; j += blockDim.x) w.fill[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      for (int k = rbeg(i); k < rend(i); ++k) atomicAdd(&w.fill[ci[k]], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int j = 0; j < n; ++j) {
        w.trp[j] = acc;
        acc += w.fill[j];
        w.fill[j] = 0;
      }
      w.trp[n] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      for (int k = rbeg(i); k < rend(i); ++k) {
        const int j = ci[k];
        const int p = w.trp[j] + atomicAdd(&w.fill[j], 1);
        w.tci[p] = i;
        w.perm[p] = k;
      }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {  // insertion sort by row (stable transpose)
      const int s = w.trp[j], e = w.trp[j + 1];
      for (int a = s + 1; a < e; ++a) {
        const int ri = w.tci[a], pk = w.perm[a];
        int b2 = a - 1;
        while (b2 >= s && w.tci[b2] > ri) {
          w.tci[b2 + 1] = w.tci[b2];
          w.perm[b2 + 1] = w.perm[b2];
          --b2;
        }
        w.tci[b2 + 1] = ri;
        w.perm[b2 + 1] = pk;
      }
    }
    // ---- preconditioning (a2, a3): exactly rounded max / sqrt / division
    for (int k = threadIdx.x; k < nnz; k += blockDim.x) w.kv[k] = val[k];
    for (int i = threadIdx.x; i < m; i += blockDim.x) w.D1[i] = 1.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) w.D2[j] = 1.0;
    __syncthreads();
    const int passes = o.ruiz_iters + (o.pock_chambolle ? 1 : 0);
    for (int it = 0; it < passes; ++it) {
      const bool pc = it >= o.ruiz_iters;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double a = 0.0;
        for (int k = rbeg(i); k < rend(i); ++k) {
          const double v = fabs(w.kv[k]);
          a = pc ? a + v : (v > a ? v : a);
        }
        w.tmpm[i] = a > 0.0 ? sqrt(a) : 1.0;
      }
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double a = 0.0;
        for (int p = w.trp[j]; p < w.trp[j + 1]; ++p) {
          const double v = fabs(w.kv[w.perm[p]]);
          a = pc ? a + v : (v > a ? v : a);
        }
        w.tmpn[j] = a > 0.0 ? sqrt(a) : 1.0;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        for (int k = rbeg(i); k < rend(i); ++k) w.kv[k] = w.kv[k] / w.tmpm[i] / w.tmpn[ci[k]];
        w.D1[i] = w.D1[i] / w.tmpm[i];
      }
      for (int j = threadIdx.x; j < n; j += blockDim.x) w.D2[j] = w.D2[j] / w.tmpn[j];
      __syncthreads();
    }
    // ---- K~^T values, arithmetic copies, transform (a4)
    double kmax = 0.0;
    for (int p = threadIdx.x; p < nnz; p += blockDim.x) {
      const double v = w.kv[w.perm[p]];
      w.ktv[p] = v;
      w.kt[p] = (T)v;
    }
    for (int k = threadIdx.x; k < nnz; k += blockDim.x) {
      w.k[k] = (T)w.kv[k];
      kmax = fmax(kmax, fabs(w.kv[k]));
    }
    double nc2[4] = {0.0, 0.0, 0.0, 0.0};  // ||c~||^2, ||q~||^2, ||c||^2, ||q||^2
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      w.cs[j] = w.D2[j] * c[j];
      w.ls[j] = l[j] / w.D2[j];
      w.us[j] = u[j] / w.D2[j];
      w.csT[j] = (T)w.cs[j];
      w.lsT[j] = (T)w.ls[j];
      w.usT[j] = (T)w.us[j];
      nc2[0] += w.cs[j] * w.cs[j];
      nc2[2] += c[j] * c[j];
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      w.qs[i] = w.D1[i] * q[i];
      w.ylos[i] = (ineq[i] ? 0.0 : -INFINITY) / w.D1[i];
      w.qsT[i] = (T)w.qs[i];
      w.yloT[i] = (T)w.ylos[i];
      nc2[1] += w.qs[i] * w.qs[i];
      nc2[3] += q[i] * q[i];
    }
    kmax = cta_max(kmax, red);
    cta_sum<4>(nc2, red);
    // ---- initialisation (a5): z = proj(0), omega, eta_hat
    const double cnorm = sqrt(nc2[2]), qnorm = sqrt(nc2[3]);
    double omega = 1.0;
    {
      const double ncs = sqrt(nc2[0]), nqs = sqrt(nc2[1]);
      if (ncs > o.eps_zero && nqs > o.eps_zero) omega = ncs / nqs;
      omega *= o.primal_importance;
    }
    double eta_hat = kmax > 0.0 ? 1.0 / kmax : 1.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      // z^0 = proj(0), or the projection of the given start (scaled space)
      const T xs0 = in.x0 ? (T)(in.x0[co + j] / w.D2[j]) : T(0);
      const T x = clampv<T>(xs0, (T)w.ls[j], (T)w.us[j]);
      w.x[0][j] = x;
      w.x0[j] = x;
      w.xs[0][j] = 0.0;
      w.xs[1][j] = 0.0;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const T lo = (T)w.ylos[i];
      const T ys0 = in.y0 ? (T)(in.y0[ro + i] / w.D1[i]) : T(0);
      const T y = ys0 > lo ? ys0 : lo;
      w.y[0][i] = y;
      w.y0[i] = y;
      w.ys[0][i] = 0.0;
      w.ys[1][i] = 0.0;
    }
    __syncthreads();
    // K's row_ptr with its end entry (the input holds the m row starts)
    int32_t *rpk = w.rpk;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) rpk[i] = i < m ? rp_in[i] : nnz;
    __syncthreads();
    cta_spmv<T>(m, rpk, ci, w.k, w.x[0], Lk, prod, cap, [&](int i, T s) { w.Kx[0][i] = s; });
    __syncthreads();
    // ---- Algorithm 1 with evaluations
    int cur = 0;
    long long k = 0, t = 0, passes_used = 0, restarts = 0, k_virt = 0;
    double sum_eta = 0.0, mu0 = INFINITY, muc_prev = INFINITY;
    int status = kRunning, ret_avg = 0;
    double kkt[2][8];
    double stall_best = INFINITY;
    int stall_cnt = 0;
    bool first_eval = true;
    long long fac_k0 = 0;
    for (;;) {
      // ---------- evaluation (at the start and every eval_every steps)
      const bool eval_now = first_eval || (k % o.eval_every == 0) || k >= iter_limit ||
                            passes_used >= pass_limit;
      if (eval_now) {
        const bool avg = sum_eta > 0.0;
        const double inv = avg ? 1.0 / sum_eta : 0.0;
        const T *x = w.x[cur], *y = w.y[cur], *Kx = w.Kx[cur];
        // K^T y (current), K x (current), K^T ys, K xs: in float64 from the
        // float64 K~ whatever T, since float32 products cannot resolve the
        // residuals of Eq. (15) below about 1e-7 of their terms (in float64
        // the step's own K x is that product already)
        double *prodd = reinterpret_cast<double *>(prod);
        const int capd = (int)(kBatchSmem / sizeof(double));
        cta_spmv<double, T>(n, w.trp, w.tci, w.ktv, y, Lt, prodd, capd, [&](int j, double s) { w.KTyd[j] = s; });
        const double *Kxd = w.Kxd;
        if constexpr (sizeof(T) == 8) Kxd = reinterpret_cast<const double *>(Kx);
        else cta_spmv<double, T>(m, rpk, ci, w.kv, x, Lk, prodd, capd, [&](int i, double s) { w.Kxd[i] = s; });
        if (avg) {
          for (int j = threadIdx.x; j < n; j += blockDim.x) w.xa[j] = (T)(w.xs[cur][j] * inv);
          for (int i = threadIdx.x; i < m; i += blockDim.x) w.ya[i] = (T)(w.ys[cur][i] * inv);
          __syncthreads();
          cta_spmv<double, T>(n, w.trp, w.tci, w.ktv, w.ya, Lt, prodd, capd, [&](int j, double s) { w.KTysd[j] = s; });
          cta_spmv<double, T>(m, rpk, ci, w.kv, w.xa, Lk, prodd, capd, [&](int i, double s) { w.Kxsd[i] = s; });
        }
        __syncthreads();
        // Eq. (15) terms for both candidates on the original problem
        double acc[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[a] = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
#pragma unroll
          for (int cnd = 0; cnd < 2; ++cnd) {
            if (cnd == 1 && !avg) break;
            const double xt = cnd == 0 ? (double)x[j] : (double)w.xa[j];
            const double kt = cnd == 0 ? w.KTyd[j] : w.KTysd[j];
            const double rc = c[j] - kt / w.D2[j];
            const double lam = lam_of(rc, l[j], u[j]);
            acc[6 * cnd + 0] += c[j] * (w.D2[j] * xt);
            acc[6 * cnd + 1] += (rc - lam) * (rc - lam);
            acc[6 * cnd + 2] += (lam > 0.0 ? l[j] * lam : 0.0) + (lam < 0.0 ? u[j] * lam : 0.0);
          }
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
#pragma unroll
          for (int cnd = 0; cnd < 2; ++cnd) {
            if (cnd == 1 && !avg) break;
            const double yt = cnd == 0 ? (double)y[i] : (double)w.ya[i];
            const double kx = cnd == 0 ? Kxd[i] : w.Kxsd[i];
            double r = q[i] - kx / w.D1[i];
            if (ineq[i]) r = r > 0.0 ? r : 0.0;
            acc[6 * cnd + 3] += r * r;
            acc[6 * cnd + 4] += q[i] * (w.D1[i] * yt);
          }
        }
        cta_sum<12>(acc, red);
        bool pass[2] = {false, false};
        for (int cnd = 0; cnd < 2; ++cnd) {
          if (cnd == 1 && !avg) break;
          const double pobj = acc[6 * cnd + 0], dobj = acc[6 * cnd + 2] + acc[6 * cnd + 4];
          const double pres = sqrt(acc[6 * cnd + 3]), dres = sqrt(acc[6 * cnd + 1]);
          const double gap = fabs(dobj - pobj);
          double *kk = kkt[cnd];
          kk[0] = pobj;
          kk[1] = dobj;
          kk[2] = gap;
          kk[3] = pres;
          kk[4] = dres;
          kk[5] = gap / (1.0 + fabs(dobj) + fabs(pobj));
          kk[6] = pres / (1.0 + qnorm);
          kk[7] = dres / (1.0 + cnorm);
          pass[cnd] = kk[5] <= o.rel_tol && kk[6] <= o.rel_tol && kk[7] <= o.rel_tol;
        }
        if (pass[0] || pass[1]) {
          status = kOptimal;
          ret_avg = pass[0] ? 0 : 1;
          break;
        }
        if (!(isfinite(kkt[0][0]) && isfinite(kkt[0][1]))) {
          status = kNumErr;
          break;
        }
        if (k >= iter_limit) {
          status = kIterLimit;
          break;
        }
        if (passes_used >= pass_limit) {
          status = kKktLimit;
          break;
        }
        if (o.stall_evals > 0) {
          // the better candidate's relative error has not dropped by 10%
          // for stall_evals evaluations: the arithmetic's floor (float32)
          const double e0 = fmax(kkt[0][5], fmax(kkt[0][6], kkt[0][7]));
          const double e1 = avg ? fmax(kkt[1][5], fmax(kkt[1][6], kkt[1][7])) : INFINITY;
          const double err = fmin(e0, e1);
          if (err < 0.9 * stall_best) {
            stall_best = err;
            stall_cnt = 0;
          } else if (++stall_cnt >= o.stall_evals) {
            status = kStalled;
            ret_avg = e1 < e0 ? 1 : 0;
            break;
          }
        }
        if (!first_eval && o.adaptive_restart && avg) {
          // restart candidate and criteria (Section 3.2)
          double d2[4] = {0.0, 0.0, 0.0, 0.0};
          for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double a0 = (double)x[j] - (double)w.x0[j], a1 = (double)w.xa[j] - (double)w.x0[j];
            d2[0] += a0 * a0;
            d2[2] += a1 * a1;
          }
          for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double a0 = (double)y[i] - (double)w.y0[i], a1 = (double)w.ya[i] - (double)w.y0[i];
            d2[1] += a0 * a0;
            d2[3] += a1 * a1;
          }
          cta_sum<4>(d2, red);
          const double rcur = sqrt(omega * d2[0] + d2[1] / omega), ravg = sqrt(omega * d2[2] + d2[3] / omega);
          const double mu_cur = cta_gap<T>(w, n, m, x, y, w.KTyd, Kxd, omega, rcur, skey, sidx, red);
          const double mu_avg = cta_gap<T>(w, n, m, w.xa, w.ya, w.KTysd, w.Kxsd, omega, ravg, skey, sidx, red);
          const int cand = o.restart_to_current ? (mu_cur < mu_avg ? 0 : 1) : 1;
          const double muc = cand == 0 ? mu_cur : mu_avg;
          bool restart = false;
          if (muc <= o.beta_suff * mu0) restart = true;
          else if (muc <= o.beta_nec * mu0 && muc > muc_prev) restart = true;
          else if ((double)t >= o.beta_art * (double)k) restart = true;
          muc_prev = muc;
          if (restart) {
            const double Dx = sqrt(cand == 0 ? d2[0] : d2[2]), Dy = sqrt(cand == 0 ? d2[1] : d2[3]);
            const double *kty0 = w.KTyd, *kx0 = Kxd;  // products at the new restart point
            if (cand == 1) {  // the average becomes the current iterate
              for (int j = threadIdx.x; j < n; j += blockDim.x) w.x[cur][j] = w.xa[j];
              for (int i = threadIdx.x; i < m; i += blockDim.x) {
                w.y[cur][i] = w.ya[i];
                w.Kx[cur][i] = (T)w.Kxsd[i];
              }
              kty0 = w.KTysd;
              kx0 = w.Kxsd;
              __syncthreads();
            }
            if (o.pw_update && Dx > o.eps_zero && Dy > o.eps_zero)
              omega = exp(o.pw_theta * log(Dy / Dx) + (1.0 - o.pw_theta) * log(omega));
            // mu_0 of the new outer loop: the new start against the old one, new omega
            const double r0 = sqrt(omega * (cand == 0 ? d2[0] : d2[2]) + (cand == 0 ? d2[1] : d2[3]) / omega);
            mu0 = cta_gap<T>(w, n, m, w.x[cur], w.y[cur], kty0, kx0, omega, r0, skey, sidx, red);
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
              w.x0[j] = w.x[cur][j];
              w.xs[cur][j] = 0.0;
            }
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
              w.y0[i] = w.y[cur][i];
              w.ys[cur][i] = 0.0;
            }
            sum_eta = 0.0;
            t = 0;
            muc_prev = INFINITY;
            restarts += 1;
            __syncthreads();
          }
        } else if (!first_eval && !o.adaptive_restart && o.pw_update &&
                   (double)(k - k_virt) >= o.beta_art * (double)k) {
          // Appendix C.2 "no restart": Algorithm 3 where the artificial
          // criterion would restart, measured from the previous update's point
          double d2[2] = {0.0, 0.0};
          for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double a = (double)x[j] - (double)w.x0[j];
            d2[0] += a * a;
          }
          for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double a = (double)y[i] - (double)w.y0[i];
            d2[1] += a * a;
          }
          cta_sum<2>(d2, red);
          const double Dx = sqrt(d2[0]), Dy = sqrt(d2[1]);
          if (Dx > o.eps_zero && Dy > o.eps_zero)
            omega = exp(o.pw_theta * log(Dy / Dx) + (1.0 - o.pw_theta) * log(omega));
          for (int j = threadIdx.x; j < n; j += blockDim.x) w.x0[j] = x[j];
          for (int i = threadIdx.x; i < m; i += blockDim.x) w.y0[i] = y[i];
          k_virt = k;
          __syncthreads();
        }
        first_eval = false;
        // Algorithm 2's factors 1 - (k+1)^-0.3, 1 + (k+1)^-0.6 (k counted from 1)
        // for the steps up to the next evaluation
        fac_k0 = k;
        for (int i = threadIdx.x; i < min(o.eval_every, kMaxEval); i += blockDim.x) {
          const double kk = (double)(k + i + 1);
          fac[0][i] = 1.0 - pow(kk + 1.0, -0.3);
          fac[1][i] = 1.0 + pow(kk + 1.0, -0.6);
        }
        __syncthreads();
      }
      // ---------- one accepted step of Algorithm 2
      double eta = eta_hat;
      bool accepted = false;
      while (!accepted) {
        if (threadIdx.x == 0) {
          s_step[0] = eta / omega;
          s_step[1] = eta * omega;
        }
        __syncthreads();
        const T tau = (T)s_step[0], sig = (T)s_step[1], et = (T)eta;
        const T *x = w.x[cur], *y = w.y[cur], *Kx = w.Kx[cur];
        const double *xs = w.xs[cur], *ys = w.ys[cur];
        T *xn = w.x[cur ^ 1], *yn = w.y[cur ^ 1], *Kxn = w.Kx[cur ^ 1];
        double *xsn = w.xs[cur ^ 1], *ysn = w.ys[cur ^ 1];
        double s3[3] = {0.0, 0.0, 0.0};
        cta_spmv<T>(n, w.trp, w.tci, w.kt, y, Lt, prod, cap, [&](int j, T g) {
          const T xj = x[j];
          const T xp = clampv<T>(xj - tau * (w.csT[j] - g), w.lsT[j], w.usT[j]);
          xn[j] = xp;
          xsn[j] = xs[j] + (double)et * (double)xp;
          const T d = xp - xj;
          s3[0] += (double)(d * d);
        });
        __syncthreads();
        cta_spmv<T>(m, rpk, ci, w.k, xn, Lk, prod, cap, [&](int i, T kxn) {
          const T kx = Kx[i], yi = y[i], lo = w.yloT[i];
          const T v = yi + sig * (w.qsT[i] - T(2) * kxn + kx);
          const T yp = v > lo ? v : lo;
          yn[i] = yp;
          Kxn[i] = kxn;
          ysn[i] = ys[i] + (double)et * (double)yp;
          const T dy = yp - yi, dk = kxn - kx;
          s3[1] += (double)(dy * dy);
          s3[2] += (double)dy * (double)dk;
        });
        cta_sum_lean<3>(s3, red);
        passes_used += 1;
        // Algorithm 2's test, in one thread
        if (threadIdx.x == 0) {
          const double num = omega * s3[0] + s3[1] / omega;
          const double den = 2.0 * fabs(s3[2]);
          const double eta_bar = den > 0.0 ? num / den : INFINITY;
          const long long idx = k - fac_k0;
          double fr, fg;
          if (idx >= 0 && idx < min(o.eval_every, kMaxEval)) {
            fr = fac[0][idx];
            fg = fac[1][idx];
          } else {
            const double kk = (double)(k + 1);
            fr = 1.0 - pow(kk + 1.0, -0.3);
            fg = 1.0 + pow(kk + 1.0, -0.6);
          }
          const double e1 = fr * eta_bar, e2 = fg * eta;
          s_step[2] = e1 < e2 ? e1 : e2;
          s_step[3] = (!isfinite(num) || isnan(eta_bar) || isnan(s3[2])) ? -1.0 : (eta <= eta_bar ? 1.0 : 0.0);
        }
        __syncthreads();
        const double eta_next = s_step[2], decision = s_step[3];
        __syncthreads();
        if (decision < 0.0) {
          status = kNumErr;
          break;
        }
        if (decision > 0.0) {
          accepted = true;
          cur ^= 1;
          sum_eta += eta;
          k += 1;
          t += 1;
        }
        eta_hat = eta_next;
        eta = eta_next;
        if (!accepted && passes_used >= pass_limit) break;
      }
      if (status != kRunning) break;
      if (!accepted) continue;  // pass limit: the evaluation reports it
    }
    // ---------- output: the returned candidate in the original space
    if (status != kOptimal && status != kStalled) ret_avg = 0;
    {
      const bool avg_out = ret_avg == 1;
      const T *x = avg_out ? w.xa : w.x[cur], *y = avg_out ? w.ya : w.y[cur];
      for (int j = threadIdx.x; j < n; j += blockDim.x) out.x[co + j] = w.D2[j] * (double)x[j];
      for (int i = threadIdx.x; i < m; i += blockDim.x) out.y[ro + i] = w.D1[i] * (double)y[i];
    }
    if (threadIdx.x == 0) {
      pdlp_result r;
      memset(&r, 0, sizeof(r));
      r.status = status;
      r.returned_average = ret_avg;
      r.iters = k;
      r.kkt_passes = passes_used;
      r.restarts = restarts;
      const double *kk = kkt[ret_avg];
      r.primal_obj = kk[0];
      r.dual_obj = kk[1];
      r.gap = kk[2];
      r.pres = kk[3];
      r.dres = kk[4];
      r.rel_gap = kk[5];
      r.rel_pres = kk[6];
      r.rel_dres = kk[7];
      out.res[b] = r;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace pdlp

// =================================================================== host

namespace pdlp {
namespace {

struct Tuned {
  bool done[2][kNumBuckets] = {};
  int lanes[2][kNumBuckets] = {};  // K lanes (low byte), K^T lanes (next byte)
};
Tuned g_tuned;
std::mutex g_tune_mu;

int bucket_of(int m, long long nnz) {
  const double len = (double)nnz / (double)(m > 0 ? m : 1);
  if (len < 8) return 0;
  if (len < 16) return 1;
  if (len < 32) return 2;
  if (len < 64) return 3;
  return 4;
}

// Candidate (K lanes, K^T lanes) per bucket, timed by the autotuner.
const int kCand[][2] = {{2, 1}, {4, 2}, {4, 4}, {8, 4}, {8, 8}, {16, 8}, {32, 16}};
constexpr int kNumCand = sizeof(kCand) / sizeof(kCand[0]);

struct DevBatch {
  DevBuf mm, nn, ro, co, zo, rp, ci, val, c, q, l, u, ineq, order, lanes, x, y, res, ctr, slab;
  DevBuf x0, y0, used;  // PDLP_FP32_REFINE: the float64 stage's starts and spent budgets
};

// PDLP_FP32_REFINE batches: the float32 stage of an LP stops at this many
// evaluations (40 steps each) without a 10% gain in its relative error
// (measured on the 4,096-LP batch to 1e-8: 50 -> 1.90 s, 20 -> 1.65 s,
// 10 -> 1.49 s; to 1e-6 1.29 -> 1.30 s)
constexpr int kBatchStallEvals = 10;

template <typename T>
cudaError_t launch_batch(const BatchIn &in, const BatchOpts &o, BatchOut out, char *slab, size_t wb, int grid,
                         int mm, int nn, long long zz, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(out.queue, 0, sizeof(unsigned), st))) return e;
  k_batch<T><<<grid, kBThreads, kBatchSmem, st>>>(in, o, out, slab, wb, mm, nn, zz);
  return cudaGetLastError();
}

template <typename T>
int solve_batch_t(int32_t count, const std::vector<int32_t> &hm, const std::vector<int32_t> &hn,
                  const std::vector<int64_t> &hzo, BatchIn in, const BatchOpts &o, BatchOut out, DevBatch &db,
                  int32_t *order_host, cudaStream_t st, std::string &why) {
  cudaError_t e;
  const int pi = sizeof(T) == 8 ? 0 : 1;
  int mm = 1, nn = 1;
  long long zz = 1;
  for (int b = 0; b < count; ++b) {
    mm = std::max(mm, hm[b]);
    nn = std::max(nn, hn[b]);
    zz = std::max<long long>(zz, hzo[b + 1] - hzo[b]);
  }
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaFuncSetAttribute(k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<T>, kBThreads, kBatchSmem))) {
    why = cudaGetErrorString(e);
    return PDLP_ERR_CUDA;
  }
  const int grid = std::max(1, std::min(count, sms * std::max(per, 1)));
  const size_t wb = work_bytes<T>(mm, nn, zz);
  char *slab = reinterpret_cast<char *>(db.slab.get(wb * (size_t)grid));
  int32_t *lanes = reinterpret_cast<int32_t *>(db.lanes.get(sizeof(int32_t) * count));
  int32_t *order = reinterpret_cast<int32_t *>(db.order.get(sizeof(int32_t) * count));
  if (!slab || !lanes || !order) {
    why = "batch workspace allocation failed";
    return PDLP_ERR_OOM;
  }
  in.lanes = lanes;
  in.order = order;
  std::vector<int> bk(count);
  for (int b = 0; b < count; ++b) bk[b] = bucket_of(hm[b], hzo[b + 1] - hzo[b]);
  std::vector<int32_t> hl(count);
  // ---- autotuner: per size bucket, time a sample of its LPs for 100 steps
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    BatchOpts ot = o;
    ot.rel_tol = 0.0;  // never stops early
    ot.iter_limit = 100;
    ot.kkt_pass_limit = 1ll << 40;
    ot.stall_evals = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int bu = 0; bu < kNumBuckets; ++bu) {
      if (g_tuned.done[pi][bu]) continue;
      std::vector<int32_t> sample;
      for (int i = 0; i < count && (int)sample.size() < grid; ++i) {
        const int b = order_host[i];
        if (bk[b] == bu) sample.push_back(b);
      }
      if (sample.empty()) continue;
      float best = 1e30f;
      int best_c = 0;
      BatchIn it = in;
      it.count = (int32_t)sample.size();
      it.x0 = it.y0 = nullptr;  // timed from cold starts with full budgets
      it.used_iters = it.used_passes = nullptr;
      if ((e = cudaMemcpyAsync(order, sample.data(), sizeof(int32_t) * sample.size(), cudaMemcpyHostToDevice, st)))
        break;
      for (int cnd = 0; cnd < kNumCand && !e; ++cnd) {
        const int32_t code = kCand[cnd][0] | (kCand[cnd][1] << 8);
        for (int b : sample) hl[b] = code;
        if ((e = cudaMemcpyAsync(lanes, hl.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st))) break;
        cudaEventRecord(e0, st);
        if ((e = launch_batch<T>(it, ot, out, slab, wb, std::min<int>(grid, (int)sample.size()), mm, nn, zz, st)))
          break;
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_c = cnd;
        }
      }
      if (e) break;
      g_tuned.lanes[pi][bu] = kCand[best_c][0] | (kCand[best_c][1] << 8);
      g_tuned.done[pi][bu] = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) {
      why = std::string("batch autotuner: ") + cudaGetErrorString(e);
      return PDLP_ERR_CUDA;
    }
    for (int b = 0; b < count; ++b) hl[b] = g_tuned.lanes[pi][bk[b]];
  }
  if ((e = cudaMemcpyAsync(lanes, hl.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(order, order_host, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st)) ||
      (e = launch_batch<T>(in, o, out, slab, wb, grid, mm, nn, zz, st)) || (e = cudaStreamSynchronize(st))) {
    why = cudaGetErrorString(e);
    return PDLP_ERR_CUDA;
  }
  return PDLP_OK;
}

template <typename T>
T *dcopy(DevBuf &b, const T *src, size_t count, cudaStream_t st, cudaError_t &e) {
  T *d = reinterpret_cast<T *>(b.get(sizeof(T) * (count ? count : 1)));
  if (!d) {
    e = cudaErrorMemoryAllocation;
    return nullptr;
  }
  if (count && !e) e = cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyDefault, st);
  return d;
}

int bfail(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

}  // namespace
}  // namespace pdlp

using namespace pdlp;

extern "C" int pdlp_solve_batch(int32_t count, const int32_t *m, const int32_t *n, const int64_t *row_off,
                                const int64_t *col_off, const int64_t *nnz_off, const int32_t *row_ptr,
                                const int32_t *col_idx, const double *val, const double *c, const double *q,
                                const double *l, const double *u, const uint8_t *ineq_mask,
                                const pdlp_options *opts, double *x_out, double *y_out, pdlp_result *res) {
  if (count < 1 || !m || !n || !row_off || !col_off || !nnz_off || !row_ptr || !col_idx || !val || !c || !q ||
      !l || !u || !ineq_mask || !opts)
    return bfail(PDLP_ERR_INVALID_ARG, "NULL argument or count < 1");
  if (opts->precision != PDLP_FP64 && opts->precision != PDLP_FP32 && opts->precision != PDLP_FP32_REFINE)
    return bfail(PDLP_ERR_INVALID_ARG, "batch precision must be PDLP_FP64, PDLP_FP32 or PDLP_FP32_REFINE");
  if (opts->eval_every < 1 || !(opts->rel_tol >= 0.0) || opts->ruiz_iters < 0)
    return bfail(PDLP_ERR_INVALID_ARG, "bad options");
  if (opts->step_policy != 0 || opts->omega0 != 0.0)
    return bfail(PDLP_ERR_INVALID_ARG, "the batched solve uses Algorithm 2 and InitializePrimalWeight only");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(opts->stream);
  cudaError_t e = cudaSuccess;
  std::vector<int32_t> hm(count), hn(count);
  std::vector<int64_t> hro(count + 1), hco(count + 1), hzo(count + 1);
  e = cudaMemcpy(hm.data(), m, sizeof(int32_t) * count, cudaMemcpyDefault);
  if (!e) e = cudaMemcpy(hn.data(), n, sizeof(int32_t) * count, cudaMemcpyDefault);
  if (!e) e = cudaMemcpy(hro.data(), row_off, sizeof(int64_t) * (count + 1), cudaMemcpyDefault);
  if (!e) e = cudaMemcpy(hco.data(), col_off, sizeof(int64_t) * (count + 1), cudaMemcpyDefault);
  if (!e) e = cudaMemcpy(hzo.data(), nnz_off, sizeof(int64_t) * (count + 1), cudaMemcpyDefault);
  if (e) return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  if (hro[0] != 0 || hco[0] != 0 || hzo[0] != 0) return bfail(PDLP_ERR_INVALID_ARG, "offsets must start at 0");
  for (int b = 0; b < count; ++b) {
    if (hm[b] < 1 || hn[b] < 1 || hro[b + 1] - hro[b] != hm[b] || hco[b + 1] - hco[b] != hn[b] ||
        hzo[b + 1] < hzo[b] || hzo[b + 1] - hzo[b] > 2147483647ll)
      return bfail(PDLP_ERR_INVALID_ARG, "LP " + std::to_string(b) + ": sizes and offsets disagree");
    if (hm[b] + hn[b] > kSortMax)
      return bfail(PDLP_ERR_INVALID_ARG, "LP " + std::to_string(b) + ": batch LPs need m + n <= 4096");
  }
  const int64_t R = hro[count], Cc = hco[count], Z = hzo[count];
  static DevBatch db;  // grown as needed; one batch call at a time per process
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  BatchIn in{};
  in.count = count;
  in.m = dcopy(db.mm, m, count, st, e);
  in.n = dcopy(db.nn, n, count, st, e);
  in.row_off = dcopy(db.ro, row_off, count + 1, st, e);
  in.col_off = dcopy(db.co, col_off, count + 1, st, e);
  in.nnz_off = dcopy(db.zo, nnz_off, count + 1, st, e);
  in.rp = dcopy(db.rp, row_ptr, R, st, e);
  in.ci = dcopy(db.ci, col_idx, Z, st, e);
  in.val = dcopy(db.val, val, Z, st, e);
  in.c = dcopy(db.c, c, Cc, st, e);
  in.q = dcopy(db.q, q, R, st, e);
  in.l = dcopy(db.l, l, Cc, st, e);
  in.u = dcopy(db.u, u, Cc, st, e);
  in.ineq = dcopy(db.ineq, ineq_mask, R, st, e);
  BatchOut out{};
  out.x = reinterpret_cast<double *>(db.x.get(sizeof(double) * Cc));
  out.y = reinterpret_cast<double *>(db.y.get(sizeof(double) * R));
  out.res = reinterpret_cast<pdlp_result *>(db.res.get(sizeof(pdlp_result) * count));
  unsigned *ctr = reinterpret_cast<unsigned *>(db.ctr.get(2 * sizeof(unsigned)));
  if (e || !out.x || !out.y || !out.res || !ctr)
    return bfail(e ? PDLP_ERR_CUDA : PDLP_ERR_OOM, e ? cudaGetErrorString(e) : "allocation failed");
  out.queue = ctr;
  out.bad = ctr + 1;
  if ((e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st))) return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  BatchOpts o{};
  o.rel_tol = opts->rel_tol;
  o.eps_zero = opts->eps_zero;
  o.beta_suff = opts->beta_suff;
  o.beta_nec = opts->beta_nec;
  o.beta_art = opts->beta_art;
  o.pw_theta = opts->pw_smoothing;
  o.primal_importance = opts->primal_importance;
  o.iter_limit = opts->iter_limit;
  o.kkt_pass_limit = opts->kkt_pass_limit;
  o.ruiz_iters = opts->ruiz_iters;
  o.pock_chambolle = opts->pock_chambolle;
  o.eval_every = opts->eval_every;
  o.adaptive_restart = opts->adaptive_restart;
  o.pw_update = opts->pw_update;
  o.restart_to_current = opts->restart_to_current;
  // largest first
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return hzo[a + 1] - hzo[a] > hzo[b + 1] - hzo[b]; });
  std::string why;
  auto check_bad = [&]() -> int {
    unsigned bad = 0;
    if ((e = cudaMemcpy(&bad, out.bad, sizeof(unsigned), cudaMemcpyDeviceToHost)))
      return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
    if (bad) return bfail(PDLP_ERR_INVALID_ARG, "LP " + std::to_string(bad - 1) +
                                                    ": invalid data (column index range or order, non-finite "
                                                    "value, or l > u)");
    return PDLP_OK;
  };
  std::vector<pdlp_result> r1;  // float32 stage of PDLP_FP32_REFINE
  int rc;
  if (opts->precision == PDLP_FP32_REFINE) {
    // float32 steps until Eq. (15) holds at max(rel_tol, inner_tol) (the
    // float32 stage aims no tighter than what float32 resolves) or the
    // float32 floor (a stall), then float64 steps from each LP's float32
    // point to rel_tol with what is left of its iteration and KKT-pass
    // budgets (an LP already solved passes the float64 check at its start)
    BatchOpts o1 = o;
    o1.rel_tol = std::max(opts->rel_tol, opts->inner_tol);
    o1.stall_evals = kBatchStallEvals;
    rc = solve_batch_t<float>(count, hm, hn, hzo, in, o1, out, db, order.data(), st, why);
    if (rc) return bfail(rc, why);
    if ((rc = check_bad())) return rc;
    r1.resize(count);
    if ((e = cudaMemcpy(r1.data(), out.res, sizeof(pdlp_result) * count, cudaMemcpyDeviceToHost)))
      return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
    std::vector<long long> used(2 * (size_t)count);
    for (int b = 0; b < count; ++b) {
      used[b] = r1[b].iters;
      used[count + b] = r1[b].kkt_passes;
    }
    double *x0 = reinterpret_cast<double *>(db.x0.get(sizeof(double) * Cc));
    double *y0 = reinterpret_cast<double *>(db.y0.get(sizeof(double) * R));
    long long *du = reinterpret_cast<long long *>(db.used.get(sizeof(long long) * 2 * count));
    if (!x0 || !y0 || !du) return bfail(PDLP_ERR_OOM, "allocation failed");
    e = cudaMemcpyAsync(x0, out.x, sizeof(double) * Cc, cudaMemcpyDeviceToDevice, st);
    if (!e) e = cudaMemcpyAsync(y0, out.y, sizeof(double) * R, cudaMemcpyDeviceToDevice, st);
    if (!e) e = cudaMemcpyAsync(du, used.data(), sizeof(long long) * 2 * count, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
    in.x0 = x0;
    in.y0 = y0;
    in.used_iters = du;
    in.used_passes = du + count;
    rc = solve_batch_t<double>(count, hm, hn, hzo, in, o, out, db, order.data(), st, why);
  } else {
    rc = opts->precision == PDLP_FP64
             ? solve_batch_t<double>(count, hm, hn, hzo, in, o, out, db, order.data(), st, why)
             : solve_batch_t<float>(count, hm, hn, hzo, in, o, out, db, order.data(), st, why);
  }
  if (rc) return bfail(rc, why);
  if ((rc = check_bad())) return rc;
  if (!r1.empty()) {
    // the float64 stage's outcome, with both stages' counts
    std::vector<pdlp_result> r2(count);
    if ((e = cudaMemcpy(r2.data(), out.res, sizeof(pdlp_result) * count, cudaMemcpyDeviceToHost)))
      return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
    for (int b = 0; b < count; ++b) {
      r2[b].iters += r1[b].iters;
      r2[b].kkt_passes += r1[b].kkt_passes;
      r2[b].restarts += r1[b].restarts;
      r2[b].refine_rounds = 1;
    }
    if (res && (e = cudaMemcpy(res, r2.data(), sizeof(pdlp_result) * count, cudaMemcpyDefault)))
      return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
    res = nullptr;  // written
  }
  if (x_out && (e = cudaMemcpy(x_out, out.x, sizeof(double) * Cc, cudaMemcpyDefault)))
    return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  if (y_out && (e = cudaMemcpy(y_out, out.y, sizeof(double) * R, cudaMemcpyDefault)))
    return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  if (res && (e = cudaMemcpy(res, out.res, sizeof(pdlp_result) * count, cudaMemcpyDefault)))
    return bfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  return PDLP_OK;
}

extern "C" int pdlp_batch_lanes(int32_t precision, int32_t *lanes_k, int32_t *lanes_kt, int32_t nbuckets) {
  if (!lanes_k || !lanes_kt || nbuckets < 1 || (precision != PDLP_FP64 && precision != PDLP_FP32))
    return bfail(PDLP_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const int pi = precision == PDLP_FP64 ? 0 : 1;
  for (int b = 0; b < nbuckets; ++b) {
    const bool ok = b < kNumBuckets && g_tuned.done[pi][b];
    lanes_k[b] = ok ? (g_tuned.lanes[pi][b] & 0xff) : 0;
    lanes_kt[b] = ok ? ((g_tuned.lanes[pi][b] >> 8) & 0xff) : 0;
  }
  return PDLP_OK;
}
