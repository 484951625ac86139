// Presolve-lite (the cheap reductions that come before PDLP's Section 3.4
// presolve step) and postsolve, as device passes:
//   * a variable with l_j = u_j is fixed at l_j: its column leaves K and
//     q_i <- q_i - K_ij l_j;
//   * a row left without nonzeros is dropped when 0 satisfies it (K_i x >= q_i
//     with q_i <= 0, or K_i x = q_i with q_i = 0, both to 1e-9 relative) with
//     y_i = 0; otherwise the LP is primal infeasible;
//   * a column without nonzeros is set at the bound its cost points to
//     (l_j for c_j > 0, u_j for c_j < 0, the point of [l_j, u_j] nearest 0
//     for c_j = 0); an infinite such bound makes the LP unbounded;
//   * inconsistent bounds (l_j > u_j) are rejected by the input validation.
// The remaining rows and columns are renumbered in their original order and
// the reduced CSR keeps each row's column order.  Postsolve expands the
// reduced solution (removed columns at their values, removed rows with
// y_i = 0) and evaluates Eq. (15) on the original problem with its own K and
// K^T (fixed-order sums).
#include <math.h>

#include <algorithm>

#include "presolve.cuh"

namespace pdlp {

namespace {

constexpr double kEmptyRowTol = 1e-9;
enum : unsigned { kFlagPrimalInf = 1u, kFlagUnbounded = 2u };

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return (int)std::max<int64_t>(g, 1);
}

template <typename T>
T *take(DevBuf &b, size_t count) {
  return reinterpret_cast<T *>(b.get(sizeof(T) * (count ? count : 1)));
}

__device__ __forceinline__ bool fixed_col(const double *l, const double *u, int j) { return l[j] == u[j]; }

// Columns: kept (free to move and with a nonzero), or removed with their value.
__global__ void k_pre_cols(int32_t n, const double *c, const double *l, const double *u, const int32_t *trp,
                           int32_t *keepc, double *xfix, unsigned *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned bad = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const bool fixed = fixed_col(l, u, (int)j);
    const bool empty = trp[j + 1] == trp[j];
    keepc[j] = (!fixed && !empty) ? 1 : 0;
    double v = NAN;
    if (fixed) {
      v = l[j];
    } else if (empty) {
      if (c[j] > 0.0) {
        v = l[j];
        if (!(v > -INFINITY)) bad |= kFlagUnbounded;
      } else if (c[j] < 0.0) {
        v = u[j];
        if (!(v < INFINITY)) bad |= kFlagUnbounded;
      } else {
        v = 0.0 < l[j] ? l[j] : (0.0 > u[j] ? u[j] : 0.0);
      }
    }
    xfix[j] = v;
  }
  if (bad) atomicOr(flags, bad);
}

// Rows, one warp each: nonzeros in free columns, q shifted by the fixed ones
// (lane-strided partial sums, then a fixed shuffle tree), feasibility of a
// row left empty.
__global__ void k_pre_rows(int32_t m, const int32_t *rp, const int32_t *ci, const double *val, const double *q,
                           const uint8_t *ineq, const double *l, const double *u, int32_t *cnt, double *qsh,
                           int32_t *keepr, unsigned *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nw) {
    double acc = 0.0;
    int c = 0;
    for (int32_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int j = ci[k];
      if (fixed_col(l, u, j)) acc += val[k] * l[j];
      else ++c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(0xffffffffu, acc, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      const double qs = q[i] - acc;
      cnt[i] = c;
      keepr[i] = c > 0 ? 1 : 0;
      qsh[i] = qs;
      if (c == 0) {
        const double tol = kEmptyRowTol * (1.0 + fabs(q[i]));
        const bool infeasible = ineq[i] ? qs > tol : fabs(qs) > tol;
        if (infeasible) atomicOr(flags, kFlagPrimalInf);
      }
    }
  }
}

// Reduced CSR, one warp per kept row: entries in free columns in their order.
__global__ void k_pre_scatter(int32_t m, const int32_t *rp, const int32_t *ci, const double *val, const double *l,
                              const double *u, const int32_t *keepr, const int32_t *rownew, const int32_t *roff,
                              const int32_t *colnew, int32_t *rp1, int32_t *ci1, double *val1) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nw) {
    if (!keepr[i]) continue;
    int base = roff[i];
    if (lane == 0) rp1[rownew[i]] = base;
    for (int32_t k0 = rp[i]; k0 < rp[i + 1]; k0 += 32) {
      const int32_t k = k0 + lane;
      const bool take_it = k < rp[i + 1] && !fixed_col(l, u, ci[k]);
      const unsigned mask = __ballot_sync(0xffffffffu, take_it);
      if (take_it) {
        const int pos = base + __popc(mask & ((1u << lane) - 1u));
        ci1[pos] = colnew[ci[k]];
        val1[pos] = val[k];
      }
      base += __popc(mask);
    }
  }
}

__global__ void k_pre_vectors(int32_t m, int32_t n, const double *c, const double *l, const double *u,
                              const double *qsh, const uint8_t *ineq, const int32_t *keepr, const int32_t *rownew,
                              const int32_t *keepc, const int32_t *colnew, double *c1, double *l1, double *u1,
                              double *q1, uint8_t *ineq1) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m + n; t += stride) {
    if (t < n) {
      const int j = (int)t;
      if (keepc[j]) {
        c1[colnew[j]] = c[j];
        l1[colnew[j]] = l[j];
        u1[colnew[j]] = u[j];
      }
    } else {
      const int i = (int)(t - n);
      if (keepr[i]) {
        q1[rownew[i]] = qsh[i];
        ineq1[rownew[i]] = ineq[i];
      }
    }
  }
}

__global__ void k_pre_map_in(int32_t m, int32_t n, const double *x0, const double *y0, const int32_t *keepr,
                             const int32_t *rownew, const int32_t *keepc, const int32_t *colnew, double *x1,
                             double *y1) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m + n; t += stride) {
    if (t < n) {
      if (keepc[t]) x1[colnew[t]] = x0 ? x0[t] : 0.0;
    } else {
      const int64_t i = t - n;
      if (keepr[i]) y1[rownew[i]] = y0 ? y0[i] : 0.0;
    }
  }
}

__global__ void k_post_expand(int32_t m, int32_t n, const double *x1, const double *y1, const int32_t *keepr,
                              const int32_t *rownew, const int32_t *keepc, const int32_t *colnew,
                              const double *xfix, double *x, double *y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m + n; t += stride) {
    if (t < n) {
      x[t] = keepc[t] ? x1[colnew[t]] : xfix[t];
    } else {
      const int64_t i = t - n;
      y[i] = keepr[i] ? y1[rownew[i]] : 0.0;
    }
  }
}

// Row sums of a CSR matrix, one warp per row (lane-strided, fixed shuffle tree).
__global__ void k_post_rowsum(int32_t rows, const int32_t *rp, const int32_t *ci, const double *val,
                              const double *v, double *out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < rows; i += nw) {
    double acc = 0.0;
    for (int32_t k = rp[i] + lane; k < rp[i + 1]; k += 32) acc += val[k] * v[ci[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc;
  }
}

__global__ void k_post_gather(int64_t nnz, const double *val, const int32_t *perm, double *tval) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) tval[p] = val[perm[p]];
}

__device__ __forceinline__ double lam_of(double rc, double l, double u) {
  const bool lf = l > -INFINITY, uf = u < INFINITY;
  if (!lf && !uf) return 0.0;
  if (!lf) return rc < 0.0 ? rc : 0.0;
  if (!uf) return rc > 0.0 ? rc : 0.0;
  return rc;
}

// Per-CTA partial sums of Eq. (15) on the original problem:
// [c^T x, dual objective, ||pres||^2, ||dres||^2, ||q||^2, ||c||^2].
__global__ void __launch_bounds__(256) k_post_terms(int32_t m, int32_t n, const double *c, const double *q,
                                                    const double *l, const double *u, const uint8_t *ineq,
                                                    const double *x, const double *y, const double *kx,
                                                    const double *kty, double *part) {
  __shared__ double red[6 * 8];
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m + n; t += stride) {
    if (t < n) {
      const double rc = c[t] - kty[t];
      const double lam = lam_of(rc, l[t], u[t]);
      acc[0] += c[t] * x[t];
      acc[1] += (lam > 0.0 ? l[t] * lam : 0.0) + (lam < 0.0 ? u[t] * lam : 0.0);
      acc[3] += (rc - lam) * (rc - lam);
      acc[5] += c[t] * c[t];
    } else {
      const int64_t i = t - n;
      double r = q[i] - kx[i];
      if (ineq[i]) r = r > 0.0 ? r : 0.0;
      acc[1] += q[i] * y[i];
      acc[2] += r * r;
      acc[4] += q[i] * q[i];
    }
  }
  block_sum<6>(acc, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 6; ++a) part[6 * blockIdx.x + a] = acc[a];
}

__global__ void __launch_bounds__(256) k_post_final(int nparts, const double *part, double *kkt) {
  __shared__ double red[6 * 8];
  double s[6];
  sum_partials<6>(part, nparts, 6, s, red);
  if (threadIdx.x == 0) {
    const double pobj = s[0], dobj = s[1], pres = sqrt(s[2]), dres = sqrt(s[3]);
    const double gap = fabs(dobj - pobj);
    kkt[0] = pobj;
    kkt[1] = dobj;
    kkt[2] = gap;
    kkt[3] = pres;
    kkt[4] = dres;
    kkt[5] = gap / (1.0 + fabs(dobj) + fabs(pobj));
    kkt[6] = pres / (1.0 + sqrt(s[4]));
    kkt[7] = dres / (1.0 + sqrt(s[5]));
  }
}

constexpr int kPostGrid = 152;

}  // namespace

cudaError_t presolve_run(Presolve &pre, cudaStream_t st) {
  cudaError_t e;
  const int32_t m = pre.m0, n = pre.n0;
  const int64_t nnz = pre.nnz0;
  const int32_t *rp = reinterpret_cast<const int32_t *>(pre.rp0.ptr());
  const int32_t *ci = reinterpret_cast<const int32_t *>(pre.ci0.ptr());
  const double *val = reinterpret_cast<const double *>(pre.val0.ptr());
  const double *c = reinterpret_cast<const double *>(pre.c0.ptr());
  const double *q = reinterpret_cast<const double *>(pre.q0.ptr());
  const double *l = reinterpret_cast<const double *>(pre.l0.ptr());
  const double *u = reinterpret_cast<const double *>(pre.u0.ptr());
  const uint8_t *ineq = reinterpret_cast<const uint8_t *>(pre.ineq0.ptr());
  // K^T of the original problem (column counts; the final evaluation)
  int32_t *trp = take<int32_t>(pre.trp0, (size_t)n + 1), *tci = take<int32_t>(pre.tci0, nnz);
  int32_t *tperm = take<int32_t>(pre.tperm0, nnz);
  double *tval = take<double>(pre.tval0, nnz);
  if (!trp || !tci || !tperm || !tval) return cudaErrorMemoryAllocation;
  if ((e = build_transpose(m, n, nnz, rp, ci, trp, tci, tperm, pre.ttmp, st))) return e;
  if (nnz > 0) k_post_gather<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, val, tperm, tval);
  // columns and rows
  int32_t *keepc = take<int32_t>(pre.colnew, 2 * (size_t)n + 2);  // [keep flags | new index]
  int32_t *keepr = take<int32_t>(pre.rownew, 3 * (size_t)m + 3);  // [keep | new index | row offset]
  int32_t *cnt = take<int32_t>(pre.cnt, (size_t)m + 1 + (size_t)scan_tmp_ints((int64_t)std::max(m, n) + 1));
  double *xfix = take<double>(pre.xfix, n), *qsh = take<double>(pre.qsh, m);
  unsigned *flags = take<unsigned>(pre.flags, 8);
  if (!keepc || !keepr || !cnt || !xfix || !qsh || !flags) return cudaErrorMemoryAllocation;
  int32_t *colnew = keepc + n + 1, *rownew = keepr + m + 1, *roff = keepr + 2 * ((size_t)m + 1);
  int *scan_tmp = cnt + m + 1;
  if ((e = cudaMemsetAsync(flags, 0, 8 * sizeof(unsigned), st))) return e;
  k_pre_cols<<<grid_for(n, 256), 256, 0, st>>>(n, c, l, u, trp, keepc, xfix, flags);
  k_pre_rows<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(m, rp, ci, val, q, ineq, l, u, cnt, qsh, keepr, flags);
  // renumbering: exclusive scans of the keep flags and of the kept rows' counts
  int *tot = reinterpret_cast<int *>(flags + 2);  // [m1, n1, nnz1]
  if ((e = exclusive_scan(keepr, m, rownew, tot + 0, scan_tmp, st))) return e;
  if ((e = exclusive_scan(keepc, n, colnew, tot + 1, scan_tmp, st))) return e;
  if ((e = exclusive_scan(cnt, m, roff, tot + 2, scan_tmp, st))) return e;
  unsigned hf[8];
  if ((e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  pre.m1 = (int32_t)hf[2];
  pre.n1 = (int32_t)hf[3];
  pre.nnz1 = (int64_t)hf[4];
  if (hf[0] & kFlagPrimalInf) pre.status = kPrimalInfeasible;
  else if (hf[0] & kFlagUnbounded) pre.status = kDualInfeasible;
  else if (pre.m1 == 0 || pre.n1 == 0) pre.status = kOptimal;
  else pre.status = kPreReduced;
  // the reduced problem
  const int32_t m1 = std::max(pre.m1, 1), n1 = std::max(pre.n1, 1);
  int32_t *rp1 = take<int32_t>(pre.rp1, (size_t)m1 + 1), *ci1 = take<int32_t>(pre.ci1, pre.nnz1);
  double *val1 = take<double>(pre.val1, pre.nnz1), *c1 = take<double>(pre.c1, n1), *l1 = take<double>(pre.l1, n1),
         *u1 = take<double>(pre.u1, n1), *q1 = take<double>(pre.q1, m1);
  uint8_t *ineq1 = take<uint8_t>(pre.ineq1, m1);
  double *x1 = take<double>(pre.x1, n1), *y1 = take<double>(pre.y1, m1);
  double *kx = take<double>(pre.kx, m), *kty = take<double>(pre.kty, n);
  double *part = take<double>(pre.part, 6 * (size_t)kPostGrid + 8);
  if (!rp1 || !ci1 || !val1 || !c1 || !l1 || !u1 || !q1 || !ineq1 || !x1 || !y1 || !kx || !kty || !part)
    return cudaErrorMemoryAllocation;
  if (pre.status == kPreReduced) {
    k_pre_scatter<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(m, rp, ci, val, l, u, keepr, rownew, roff, colnew,
                                                                   rp1, ci1, val1);
    const int32_t end = (int32_t)pre.nnz1;
    if ((e = cudaMemcpyAsync(rp1 + pre.m1, &end, sizeof(int32_t), cudaMemcpyHostToDevice, st))) return e;
    k_pre_vectors<<<grid_for((int64_t)m + n, 256), 256, 0, st>>>(m, n, c, l, u, qsh, ineq, keepr, rownew, keepc,
                                                                  colnew, c1, l1, u1, q1, ineq1);
  }
  if ((e = cudaGetLastError())) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t presolve_map_start(Presolve &pre, const double *x0, const double *y0, cudaStream_t st) {
  const int32_t m = pre.m0, n = pre.n0;
  const int32_t *keepc = reinterpret_cast<const int32_t *>(pre.colnew.ptr()), *colnew = keepc + n + 1;
  const int32_t *keepr = reinterpret_cast<const int32_t *>(pre.rownew.ptr()), *rownew = keepr + m + 1;
  k_pre_map_in<<<grid_for((int64_t)m + n, 256), 256, 0, st>>>(m, n, x0, y0, keepr, rownew, keepc, colnew,
                                                               reinterpret_cast<double *>(pre.x1.ptr()),
                                                               reinterpret_cast<double *>(pre.y1.ptr()));
  return cudaGetLastError();
}

cudaError_t postsolve(Presolve &pre, const double *x1, const double *y1, double *x, double *y, double *kkt,
                      cudaStream_t st) {
  cudaError_t e;
  const int32_t m = pre.m0, n = pre.n0;
  const int32_t *keepc = reinterpret_cast<const int32_t *>(pre.colnew.ptr()), *colnew = keepc + n + 1;
  const int32_t *keepr = reinterpret_cast<const int32_t *>(pre.rownew.ptr()), *rownew = keepr + m + 1;
  k_post_expand<<<grid_for((int64_t)m + n, 256), 256, 0, st>>>(m, n, x1, y1, keepr, rownew, keepc, colnew,
                                                                reinterpret_cast<const double *>(pre.xfix.ptr()), x,
                                                                y);
  double *kx = reinterpret_cast<double *>(pre.kx.ptr()), *kty = reinterpret_cast<double *>(pre.kty.ptr());
  k_post_rowsum<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(
      m, reinterpret_cast<const int32_t *>(pre.rp0.ptr()), reinterpret_cast<const int32_t *>(pre.ci0.ptr()),
      reinterpret_cast<const double *>(pre.val0.ptr()), x, kx);
  k_post_rowsum<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(
      n, reinterpret_cast<const int32_t *>(pre.trp0.ptr()), reinterpret_cast<const int32_t *>(pre.tci0.ptr()),
      reinterpret_cast<const double *>(pre.tval0.ptr()), y, kty);
  double *part = reinterpret_cast<double *>(pre.part.ptr());
  k_post_terms<<<kPostGrid, 256, 0, st>>>(
      m, n, reinterpret_cast<const double *>(pre.c0.ptr()), reinterpret_cast<const double *>(pre.q0.ptr()),
      reinterpret_cast<const double *>(pre.l0.ptr()), reinterpret_cast<const double *>(pre.u0.ptr()),
      reinterpret_cast<const uint8_t *>(pre.ineq0.ptr()), x, y, kx, kty, part);
  k_post_final<<<1, 256, 0, st>>>(kPostGrid, part, part + 6 * kPostGrid);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(kkt, part + 6 * kPostGrid, 8 * sizeof(double), cudaMemcpyDeviceToHost, st))) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace pdlp
