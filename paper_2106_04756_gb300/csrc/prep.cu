// Create-time kernels: input validation, the stable CSR transpose that builds
// K^T, the diagonal preconditioning of Section 3.5 (Ruiz, then Pock-Chambolle
// with alpha = 1), the transform of (c, q, l, u) and the row-block schedule.
//
// Bit-exactness: every floating-point operation here is a single correctly
// rounded IEEE operation (max, abs, sqrt, division, multiplication, addition
// in a fixed sequential order), written with the _rn intrinsics so that the
// compiler cannot contract or reorder them.  The results therefore equal those
// of any sequential IEEE implementation of the same formulas.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "prep.cuh"

namespace pdlp {

// ------------------------------------------------------------- validation

// Error bits written by k_validate.
enum : unsigned { kBadRowPtr = 1u, kBadCol = 2u, kUnsorted = 4u, kBadVal = 8u, kBadBounds = 16u,
                  kBadCost = 32u, kBadRhs = 64u };

__global__ void k_validate(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                           const double *val, const double *c, const double *q, const double *l,
                           const double *u, unsigned *err) {
  unsigned bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0 && (rp[0] != 0 || (int64_t)rp[m] != nnz)) bad |= kBadRowPtr;
  for (int64_t i = tid; i < m; i += stride) {
    const int32_t s = rp[i], e = rp[i + 1];
    if (e < s || s < 0 || (int64_t)e > nnz) { bad |= kBadRowPtr; continue; }
    if (!isfinite(q[i])) bad |= kBadRhs;
  }
  for (int64_t k = tid; k < nnz; k += stride) {
    const int32_t j = ci[k];
    if (j < 0 || j >= n) bad |= kBadCol;
    if (!isfinite(val[k])) bad |= kBadVal;
  }
  for (int64_t j = tid; j < n; j += stride) {
    if (!isfinite(c[j])) bad |= kBadCost;
    if (!(l[j] <= u[j]) || l[j] == INFINITY || u[j] == -INFINITY || isnan(l[j]) || isnan(u[j]))
      bad |= kBadBounds;
  }
  if (bad) atomicOr(err, bad);
}

// Row index of every nonzero (one warp per row, lanes strided: a long row
// is written by its warp with coalesced stores).  Needs a valid row_ptr.
// rowid[k]: the row holding nonzero k, by a binary search of the (valid)
// row starts per nonzero, so that a row of a million entries is spread over
// the grid like any other
__global__ void k_row_ids(int32_t m, int64_t nnz, const int32_t *rp, int32_t *rowid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
    int32_t lo = 0, hi = m;  // the last row with rp[row] <= k
    while (hi - lo > 1) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (rp[mid] <= k) lo = mid; else hi = mid;
    }
    rowid[k] = lo;
  }
}

// Column indices strictly increasing within each row: one check per nonzero.
__global__ void k_validate_sorted(int64_t nnz, const int32_t *rowid, const int32_t *ci, unsigned *err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned bad = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; k < nnz; k += stride)
    if (rowid[k] == rowid[k - 1] && ci[k] <= ci[k - 1]) bad = kUnsorted;
  if (bad) atomicOr(err, bad);
}

const char *validate_message(unsigned bits) {
  if (bits & kBadRowPtr) return "row_ptr must start at 0, be non-decreasing and end at nnz";
  if (bits & kBadCol) return "col_idx out of range [0, n)";
  if (bits & kUnsorted) return "col_idx must be strictly increasing within each row";
  if (bits & kBadVal) return "K has a non-finite value";
  if (bits & kBadBounds) return "bounds must satisfy l <= u, l != +inf, u != -inf";
  if (bits & kBadCost) return "c has a non-finite entry";
  if (bits & kBadRhs) return "q has a non-finite entry";
  return "invalid input";
}

// ------------------------------------------------------------------ scans

// Exclusive prefix sum of int32 counts (n entries) into out (n entries) and
// total in *total; three phases, single-pass-per-phase, deterministic.
constexpr int kScanThreads = 1024, kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_excl_scan_int(int v, int *sh, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int before = warp > 0 ? sh[warp - 1] : 0;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_tiles(const int *in, int64_t n, int *tile_sum) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int a = 0; a < kScanItems; ++a) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + a;
    if (i < n) s += in[i];
  }
  int tot;
  block_excl_scan_int(s, sh, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int *tile_sum, int ntiles, int *total) {
  __shared__ int sh[32];
  int carry = 0;
  for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const int v = b < ntiles ? tile_sum[b] : 0;
    int tot;
    const int ex = block_excl_scan_int(v, sh, &tot);
    if (b < ntiles) tile_sum[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const int *in, int64_t n, const int *tile_off, int *out) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int v[kScanItems], s = 0;
  for (int a = 0; a < kScanItems; ++a) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + a;
    v[a] = i < n ? in[i] : 0;
    s += v[a];
  }
  int tot;
  int ex = block_excl_scan_int(s, sh, &tot) + tile_off[blockIdx.x];
  for (int a = 0; a < kScanItems; ++a) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + a;
    if (i < n) out[i] = ex;
    ex += v[a];
  }
}

cudaError_t exclusive_scan(const int *in, int64_t n, int *out, int *total, int *tmp, cudaStream_t st) {
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  if (ntiles == 0) return cudaMemsetAsync(total, 0, sizeof(int), st);
  k_scan_tiles<<<ntiles, kScanThreads, 0, st>>>(in, n, tmp);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(tmp, ntiles, total);
  k_scan_apply<<<ntiles, kScanThreads, 0, st>>>(in, n, tmp, out);
  return cudaGetLastError();
}

int64_t scan_tmp_ints(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// -------------------------------------------------------------- transpose
//
// K^T is K's entries stably sorted by column (so rows stay increasing within
// each column).  LSD radix sort on the column index, 8 bits per pass; each
// pass is a stable counting sort: per-tile digit histograms, one exclusive
// scan over the digit-major [digit][tile] table, and a scatter in which an
// entry's rank inside its tile comes from warp match masks.

constexpr int kSortThreads = 256, kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // entries per tile
constexpr int kDigits = 256;

__global__ void k_sort_hist(const int32_t *keys, int64_t nnz, int shift, int ntiles, int *hist) {
  __shared__ int h[kDigits];
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < nnz) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void k_sort_scatter(const int32_t *keys, const int32_t *vals, int64_t nnz, int shift,
                               int ntiles, const int *offs, int32_t *keys_out, int32_t *vals_out) {
  __shared__ int base[kDigits];
  __shared__ int wcnt[kSortThreads / 32][kDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) base[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    for (int e = threadIdx.x; e < (kSortThreads / 32) * kDigits; e += blockDim.x) (&wcnt[0][0])[e] = 0;
    __syncthreads();
    const int64_t i = tbase + (int64_t)r * kSortThreads + threadIdx.x;
    const bool ok = i < nnz;
    const int32_t key = ok ? keys[i] : 0;
    const int d = ok ? ((key >> shift) & 0xff) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      int pos = base[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      keys_out[pos] = key;
      vals_out[pos] = vals[i];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kDigits; dd += blockDim.x) {
      int s = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) s += wcnt[w][dd];
      base[dd] += s;
    }
    __syncthreads();
  }
}

__global__ void k_iota(int32_t *v, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] = (int32_t)i;
}

__global__ void k_col_count(const int32_t *ci, int64_t nnz, int *cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
    atomicAdd(cnt + ci[k], 1);
}

// row of each CSR position by binary search in row_ptr; fills K^T col_idx.
__global__ void k_rows_of(const int32_t *rp, int32_t m, const int32_t *perm, int64_t nnz, int32_t *tci) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride) {
    const int32_t k = perm[t];
    int32_t lo = 0, hi = m;  // find the last row with rp[row] <= k
    while (hi - lo > 1) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (rp[mid] <= k) lo = mid; else hi = mid;
    }
    tci[t] = lo;
  }
}

template <typename T>
__global__ void k_gather(const T *src, const int32_t *perm, int64_t nnz, T *dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride) dst[t] = src[perm[t]];
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return (int)std::max<int64_t>(g, 1);
}

cudaError_t build_transpose(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                            int32_t *trp, int32_t *tci, int32_t *perm, DevBuf &tmp, cudaStream_t st) {
  cudaError_t e;
  // column counts -> K^T row_ptr
  int *cnt = reinterpret_cast<int *>(tmp.get(sizeof(int) * ((size_t)n + 1) +
                                             sizeof(int) * (size_t)scan_tmp_ints(n + 1)));
  if (!cnt) return cudaErrorMemoryAllocation;
  int *scan_tmp = cnt + n + 1;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)n + 1), st))) return e;
  if (nnz > 0) k_col_count<<<grid_for(nnz, 256), 256, 0, st>>>(ci, nnz, cnt);
  if ((e = exclusive_scan(cnt, n + 1, trp, trp + n, scan_tmp, st))) return e;
  if (nnz == 0) return cudaGetLastError();
  // radix sort (key = column, value = CSR position)
  const int ntiles = (int)((nnz + kSortTile - 1) / kSortTile);
  const int64_t hist_n = (int64_t)kDigits * ntiles;
  DevBuf sortbuf;
  size_t bytes = sizeof(int32_t) * (size_t)nnz * 4 + sizeof(int) * (size_t)hist_n * 2 +
                 sizeof(int) * (size_t)scan_tmp_ints(hist_n) + 64;
  char *p = reinterpret_cast<char *>(sortbuf.get(bytes));
  if (!p) return cudaErrorMemoryAllocation;
  int32_t *ka = reinterpret_cast<int32_t *>(p), *kb = ka + nnz, *va = kb + nnz, *vb = va + nnz;
  int *hist = reinterpret_cast<int *>(vb + nnz), *offs = hist + hist_n, *stmp = offs + hist_n;
  if ((e = cudaMemcpyAsync(ka, ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st))) return e;
  k_iota<<<grid_for(nnz, 256), 256, 0, st>>>(va, nnz);
  int bits = 0;
  while ((1ll << bits) < (int64_t)n) ++bits;
  const int passes = std::max(1, (bits + 7) / 8);
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    k_sort_hist<<<ntiles, kSortThreads, 0, st>>>(ka, nnz, shift, ntiles, hist);
    if ((e = exclusive_scan(hist, hist_n, offs, stmp + scan_tmp_ints(hist_n) - 1, stmp, st))) return e;
    k_sort_scatter<<<ntiles, kSortThreads, 0, st>>>(ka, va, nnz, shift, ntiles, offs, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if ((e = cudaMemcpyAsync(perm, va, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st))) return e;
  k_rows_of<<<grid_for(nnz, 256), 256, 0, st>>>(rp, m, perm, nnz, tci);
  if ((e = cudaGetLastError())) return e;
  return cudaStreamSynchronize(st);  // sortbuf is freed on return
}

// ------------------------------------------------------ Section 3.5 scaling

// Ruiz: r_i = max_j |K~_ij| over the row (any order gives the same maximum).
// Largest |value| of each row, four lanes per row (rows of a few nonzeros
// keep every lane busy; a maximum is exact in any order); rows longer than
// kMaxSeg get 0 here and their maximum from k_row_absmax_long.
constexpr int kMaxLanes = 4;
__global__ void k_row_absmax(int32_t rows, const int32_t *rp, const double *val, double *out) {
  const int sub = threadIdx.x & (kMaxLanes - 1);
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kMaxLanes;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / kMaxLanes;
  const int64_t iters = (rows + ng - 1) / ng;  // the same count in every lane (full-warp shuffles)
  for (int64_t t = 0; t < iters; ++t) {
    const int64_t i = grp + t * ng;
    double mx = 0.0;
    if (i < rows) {
      const int32_t k0 = rp[i], k1 = rp[i + 1];
      if (k1 - k0 <= kMaxSeg)
        for (int32_t k = k0 + sub; k < k1; k += kMaxLanes) mx = fmax(mx, fabs(val[k]));
    }
#pragma unroll
    for (int o = kMaxLanes / 2; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o, kMaxLanes));
    if (sub == 0 && i < rows) out[i] = mx;
  }
}

// One CTA per segment of a long row: the segment's largest |value| merged
// into out[row] by an atomic maximum on the bits (values are finite and
// nonnegative, where the bit order is the numeric order).
__global__ void k_row_absmax_long(const ScanSeg *segs, const double *val, double *out) {
  __shared__ double red[32];
  const ScanSeg g = segs[blockIdx.x];
  double mx = 0.0;
  for (int32_t k = g.k0 + threadIdx.x; k < g.k1; k += blockDim.x) mx = fmax(mx, fabs(val[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0)
      atomicMax(reinterpret_cast<unsigned long long *>(out + g.row), (unsigned long long)__double_as_longlong(mx));
  }
}

// Pock-Chambolle alpha = 1: r_i = sum_j |K~_ij| accumulated sequentially in CSR
// order (the order of a plain loop over the row); rows longer than kLongScan
// are left to the host (pock_chambolle).
__global__ void k_row_abssum_seq(int32_t rows, const int32_t *rp, const double *val, double *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += stride) {
    const int32_t k0 = rp[i], k1 = rp[i + 1];
    if (k1 - k0 > kLongScan) continue;
    double s = 0.0;
    for (int32_t k = k0; k < k1; ++k) s = __dadd_rn(s, fabs(val[k]));
    out[i] = s;
  }
}

// norms -> divisors: sqrt(norm), or 1 for an empty (zero) row / column; D /= divisor.
__global__ void k_norm_to_div(int32_t len, double *nrm, double *D) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    const double v = nrm[i];
    const double d = v > 0.0 ? __dsqrt_rn(v) : 1.0;
    nrm[i] = d;
    D[i] = __ddiv_rn(D[i], d);
  }
}

// K~_ij <- (K~_ij / a_i) / b_j, one thread per nonzero (rowid: row of each).
__global__ void k_scale_nnz(int64_t nnz, const int32_t *rowid, const int32_t *ci, double *val, const double *a,
                            const double *b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
    val[k] = __ddiv_rn(__ddiv_rn(val[k], a[rowid[k]]), b[ci[k]]);
}

__global__ void k_fill(double *v, int64_t n, double x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] = x;
}

cudaError_t ruiz(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci, const int32_t *rowid,
                 double *val, const int32_t *trp, double *tval, const int32_t *perm, int ruiz_iters, double *D1,
                 double *D2, double *rbuf, double *cbuf, const ScanSeg *dsegK, int nsegK, const ScanSeg *dsegKT,
                 int nsegKT, cudaStream_t st) {
  const int gz = grid_for(nnz, 256);
  const int gm = grid_for(m, 256), gn = grid_for(n, 256);
  const int gmw = grid_for((int64_t)m * kMaxLanes, 256), gnw = grid_for((int64_t)n * kMaxLanes, 256);
  k_fill<<<gm, 256, 0, st>>>(D1, m, 1.0);
  k_fill<<<gn, 256, 0, st>>>(D2, n, 1.0);
  if (nnz > 0) k_gather<double><<<gz, 256, 0, st>>>(val, perm, nnz, tval);
  for (int it = 0; it < ruiz_iters; ++it) {
    k_row_absmax<<<gmw, 256, 0, st>>>(m, rp, val, rbuf);
    k_row_absmax<<<gnw, 256, 0, st>>>(n, trp, tval, cbuf);
    if (nsegK > 0) k_row_absmax_long<<<nsegK, 256, 0, st>>>(dsegK, val, rbuf);
    if (nsegKT > 0) k_row_absmax_long<<<nsegKT, 256, 0, st>>>(dsegKT, tval, cbuf);
    k_norm_to_div<<<gm, 256, 0, st>>>(m, rbuf, D1);
    k_norm_to_div<<<gn, 256, 0, st>>>(n, cbuf, D2);
    if (nnz > 0) k_scale_nnz<<<gz, 256, 0, st>>>(nnz, rowid, ci, val, rbuf, cbuf);
    if (nnz > 0) k_gather<double><<<gz, 256, 0, st>>>(val, perm, nnz, tval);
  }
  return cudaGetLastError();
}

cudaError_t pock_chambolle(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                           const int32_t *rowid, double *val, const int32_t *trp, double *tval,
                           const int32_t *perm, double *D1, double *D2, double *rbuf, double *cbuf,
                           const PrecondPlan &pp, const int32_t *hrp, const int32_t *htrp, cudaStream_t st) {
  cudaError_t e;
  const int gz = grid_for(nnz, 256);
  const int gm = grid_for(m, 256), gn = grid_for(n, 256);
  // l1 sums of the long rows on the host, in CSR order, from the values Ruiz left
  std::vector<double> sK(pp.longK.size()), sKT(pp.longKT.size());
  if (!pp.longK.empty() || !pp.longKT.empty()) {
    if ((e = cudaStreamSynchronize(st))) return e;
    std::vector<double> buf;
    auto host_sums = [&](const std::vector<int32_t> &rows, const int32_t *hr, const double *dv,
                         std::vector<double> &out) -> cudaError_t {
      for (size_t r = 0; r < rows.size(); ++r) {
        const int32_t k0 = hr[rows[r]], k1 = hr[rows[r] + 1];
        buf.resize((size_t)(k1 - k0));
        cudaError_t e2 = cudaMemcpy(buf.data(), dv + k0, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost);
        if (e2) return e2;
        double acc = 0.0;
        for (double v : buf) acc += fabs(v);
        out[r] = acc;
      }
      return cudaSuccess;
    };
    if ((e = host_sums(pp.longK, hrp, val, sK))) return e;
    if ((e = host_sums(pp.longKT, htrp, tval, sKT))) return e;
  }
  k_row_abssum_seq<<<gm, 256, 0, st>>>(m, rp, val, rbuf);
  k_row_abssum_seq<<<gn, 256, 0, st>>>(n, trp, tval, cbuf);
  // pageable sources: each copy is staged before the call returns
  for (size_t r = 0; r < sK.size(); ++r)
    if ((e = cudaMemcpyAsync(rbuf + pp.longK[r], &sK[r], sizeof(double), cudaMemcpyHostToDevice, st))) return e;
  for (size_t r = 0; r < sKT.size(); ++r)
    if ((e = cudaMemcpyAsync(cbuf + pp.longKT[r], &sKT[r], sizeof(double), cudaMemcpyHostToDevice, st))) return e;
  k_norm_to_div<<<gm, 256, 0, st>>>(m, rbuf, D1);
  k_norm_to_div<<<gn, 256, 0, st>>>(n, cbuf, D2);
  if (nnz > 0) k_scale_nnz<<<gz, 256, 0, st>>>(nnz, rowid, ci, val, rbuf, cbuf);
  if (nnz > 0) k_gather<double><<<gz, 256, 0, st>>>(val, perm, nnz, tval);
  return cudaGetLastError();
}

// c~ = D2 c, l~ = l / D2, u~ = u / D2, q~ = D1 q, ylo~ = ylo / D1
__global__ void k_transform_cols(int32_t n, const double *D2, const double *c, const double *l,
                                 const double *u, double *cs, double *ls, double *us) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    cs[j] = __dmul_rn(D2[j], c[j]);
    ls[j] = __ddiv_rn(l[j], D2[j]);
    us[j] = __ddiv_rn(u[j], D2[j]);
  }
}
__global__ void k_transform_rows(int32_t m, const double *D1, const double *q, const double *ylo,
                                 double *qs, double *ylos) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    qs[i] = __dmul_rn(D1[i], q[i]);
    ylos[i] = __ddiv_rn(ylo[i], D1[i]);
  }
}

cudaError_t transform(int32_t m, int32_t n, const double *D1, const double *D2, const double *c,
                      const double *q, const double *l, const double *u, const double *ylo,
                      double *cs, double *qs, double *ls, double *us, double *ylos, cudaStream_t st) {
  k_transform_cols<<<grid_for(n, 256), 256, 0, st>>>(n, D2, c, l, u, cs, ls, us);
  k_transform_rows<<<grid_for(m, 256), 256, 0, st>>>(m, D1, q, ylo, qs, ylos);
  return cudaGetLastError();
}

// y lower bounds of the paper's Y: 0 on inequality rows, -inf on equality rows
__global__ void k_ylo_from_mask(int32_t m, const uint8_t *ineq, double *ylo) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    ylo[i] = ineq[i] ? 0.0 : -INFINITY;
}

cudaError_t ylo_from_mask(int32_t m, const uint8_t *ineq, double *ylo, cudaStream_t st) {
  k_ylo_from_mask<<<grid_for(m, 256), 256, 0, st>>>(m, ineq, ylo);
  return cudaGetLastError();
}

__global__ void k_to_float(const double *src, int64_t n, float *dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (float)src[i];
}

cudaError_t to_float(const double *src, int64_t n, float *dst, cudaStream_t st) {
  if (n > 0) k_to_float<<<grid_for(n, 256), 256, 0, st>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t validate(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                     const double *val, const double *c, const double *q, const double *l,
                     const double *u, int32_t *rowid, unsigned *derr, unsigned *herr, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(derr, 0, sizeof(unsigned), st))) return e;
  const int64_t big = std::max<int64_t>(std::max<int64_t>(m, n), nnz);
  k_validate<<<grid_for(big, 256), 256, 0, st>>>(m, n, nnz, rp, ci, val, c, q, l, u, derr);
  if ((e = cudaMemcpyAsync(herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  if (*herr & kBadRowPtr) return cudaSuccess;
  if (nnz > 0) k_row_ids<<<grid_for(nnz, 256), 256, 0, st>>>(m, nnz, rp, rowid);
  if (nnz > 1) k_validate_sorted<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, rowid, ci, derr);
  if ((e = cudaMemcpyAsync(herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st))) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace pdlp
