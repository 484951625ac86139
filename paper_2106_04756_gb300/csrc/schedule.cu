// Host-side planning (declared in schedule.h): plain C++ with no CUDA
// headers, compiled into the library and, by the CPU tests, on its own.
#include "schedule.h"

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

namespace pdlp {

void build_schedule(int32_t rows, const int32_t *rp, std::vector<Chunk> &chunks, std::vector<LongRow> &longrows,
                    int32_t &nseg_total) {
  chunks.clear();
  longrows.clear();
  nseg_total = 0;
  int32_t r = 0;
  while (r < rows) {
    const int32_t len = rp[r + 1] - rp[r];
    if (len > kSegNnz) {  // split across warps
      LongRow L;
      L.row = r;
      L.nseg = (len + kSegNnz - 1) / kSegNnz;
      L.part_off = nseg_total;
      L.pad = 0;
      const int32_t lr = (int32_t)longrows.size();
      longrows.push_back(L);
      for (int32_t s = 0; s < L.nseg; ++s) {
        Chunk c;
        c.row_begin = r;
        c.row_end = -(lr + 1);
        c.nnz_begin = rp[r] + s * kSegNnz;
        c.nnz_end = std::min(rp[r + 1], c.nnz_begin + kSegNnz);
        chunks.push_back(c);
      }
      nseg_total += L.nseg;
      ++r;
      continue;
    }
    if (len > kChunkNnz) {  // one warp loops over the row (only if kSegNnz > kChunkNnz)
      chunks.push_back(Chunk{r, r + 1, rp[r], rp[r + 1]});
      ++r;
      continue;
    }
    int32_t e = r;
    while (e < rows && e - r < kChunkRows) {
      if (rp[e + 1] - rp[e] > kChunkNnz) break;
      if (rp[e + 1] - rp[r] > kChunkNnz) break;
      ++e;
    }
    chunks.push_back(Chunk{r, e, rp[r], rp[e]});
    r = e;
  }
}

void build_slabs(int32_t rows, const int32_t *rp, std::vector<int32_t> &first_row, std::vector<int32_t> &head_split,
                 std::vector<int32_t> &tail_split, std::vector<SplitRow> &splits, int32_t &nparts) {
  const int64_t nnz = rp[rows];
  const int32_t nslab = (int32_t)(nnz / kSlabNnz + 1);
  first_row.assign((size_t)nslab + 1, rows);
  head_split.assign((size_t)nslab, -1);
  tail_split.assign((size_t)nslab, -1);
  splits.clear();
  nparts = 0;
  // first_row[s]: first row whose start position is >= kSlabNnz s (rows of
  // slab s start in [kSlabNnz s, kSlabNnz (s + 1)); the last slab also owns
  // the empty rows at position nnz)
  int32_t r = 0;
  for (int32_t s = 0; s < nslab; ++s) {
    const int64_t pos = (int64_t)s * kSlabNnz;
    while (r < rows && rp[r] < pos) ++r;
    first_row[s] = r;
  }
  first_row[nslab] = rows;
  for (int32_t i = 0; i < rows; ++i) {
    const int64_t b = rp[i], e = rp[i + 1];
    if (e <= b) continue;
    const int32_t sf = (int32_t)(b / kSlabNnz), sl = (int32_t)((e - 1) / kSlabNnz);
    if (sf == sl) continue;
    if (sl == sf + 1) {  // extended: the start slab reads the remainder
      tail_split[sf] = kSlabExtend - i;
      head_split[sl] = kSlabSkip;
      continue;
    }
    const int32_t id = (int32_t)splits.size();
    splits.push_back(SplitRow{i, sf, sl, nparts});
    nparts += sl - sf + 1;
    tail_split[sf] = id;
    for (int32_t s = sf + 1; s <= sl; ++s) head_split[s] = id;
  }
}

double chunk_cost(const Chunk &c, const int32_t *rp) {
  const int nnz = c.nnz_end - c.nnz_begin;
  if (c.row_end < 0) return nnz / 32.0 + 2.0 * 13.0 + 30.0;
  const int nrows = c.row_end - c.row_begin;
  int L = 32, lg = 5;
  while (L > 1 && L * nrows > 32) {
    L >>= 1;
    --lg;
  }
  unsigned best = 0;
  for (int r = c.row_begin; r < c.row_end; ++r) best = std::max(best, (unsigned)(rp[r + 1] - rp[r] + L - 1) >> lg);
  for (unsigned th = 16; th <= 128; th <<= 1) {
    unsigned ms = 0, lc = 0;
    for (int r = c.row_begin; r < c.row_end; ++r) {
      const unsigned len = (unsigned)(rp[r + 1] - rp[r]);
      if (len > th) lc += ((len + 31u) >> 5) + 5u;
      else ms = std::max(ms, (len + (unsigned)L - 1u) >> lg);
    }
    best = std::min(best, ms + lc);
  }
  // float64 chunks above 16 steps take the segmented sum (about 16 steps)
  const unsigned steps = std::min(best + (unsigned)lg, kSegStepsHost);
  return nnz / 32.0 + 2.0 * steps + 10.0;
}

void assign_chunks(const std::vector<Chunk> &chunks, const int32_t *rp, int nw, int warps_per_cta,
                   std::vector<int32_t> &idx, std::vector<int32_t> &off, int &cmax) {
  const int n = (int)chunks.size();
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) cost[i] = chunk_cost(chunks[i], rp);
  std::vector<int32_t> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  const int grid = std::max(nw / warps_per_cta, 1);
  std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<>> heap;
  for (int r = 0; r < nw; ++r) heap.push({0.0, r});
  std::vector<int32_t> owner(n);
  for (int i : order) {
    const auto top = heap.top();
    heap.pop();
    const int r = top.second;
    owner[i] = (r % grid) * warps_per_cta + r / grid;
    heap.push({top.first + cost[i], r});
  }
  off.assign((size_t)nw + 1, 0);
  for (int i = 0; i < n; ++i) ++off[owner[i] + 1];
  cmax = 0;
  for (int w = 0; w < nw; ++w) {
    cmax = std::max(cmax, off[w + 1]);
    off[w + 1] += off[w];
  }
  idx.assign((size_t)n, 0);
  std::vector<int32_t> fill(off.begin(), off.end() - 1);
  for (int i = 0; i < n; ++i) idx[fill[owner[i]]++] = i;  // each list in chunk order
}

void refine_scales(double pv, double dv, double dmax, double *dP, double *dD) {
  double P = pv > 1.0 / dmax ? 1.0 / pv : dmax;
  double D = dv > 1.0 / dmax ? 1.0 / dv : dmax;
  *dP = P < 1.0 ? 1.0 : P;
  *dD = D < 1.0 ? 1.0 : D;
}

void plan_precondition(int32_t m, const int32_t *hrp, int32_t n, const int32_t *htrp, PrecondPlan &pp) {
  auto scan = [](int32_t rows, const int32_t *rp, std::vector<ScanSeg> &segs, std::vector<int32_t> &longr) {
    segs.clear();
    longr.clear();
    for (int32_t i = 0; i < rows; ++i) {
      const int32_t k0 = rp[i], k1 = rp[i + 1];
      if (k1 - k0 <= kMaxSeg) continue;
      if (k1 - k0 > kLongScan) longr.push_back(i);
      for (int32_t k = k0; k < k1; k += kMaxSeg) segs.push_back(ScanSeg{i, k, k1 - k > kMaxSeg ? k + kMaxSeg : k1, 0});
    }
  };
  scan(m, hrp, pp.segK, pp.longK);
  scan(n, htrp, pp.segKT, pp.longKT);
}

int refine_finish_now(int round, double prev, double rel, int max_rounds) {
  if (round >= max_rounds) return 1;
  return round >= 1 && !(rel * kRefineMinGain <= prev) ? 1 : 0;
}

int refine_remaining(long long iter_limit, long long kkt_limit, double time_limit_s, long long iters,
                     long long passes, double secs, long long out[3]) {
  out[0] = iter_limit - iters;
  out[1] = kkt_limit - passes;
  out[2] = 0;
  if (out[0] <= 0) return 1;
  if (out[1] <= 0) return 2;
  if (time_limit_s > 0.0) {
    const double left = time_limit_s - secs;
    if (!(left > 0.0)) return 3;
    out[2] = (long long)(left * 1e9) > 0 ? (long long)(left * 1e9) : 1;
  }
  return 0;
}

double refine_round_tol(double rel, double tol, double inner_tol) {
  const double want = 0.1 * tol / rel;
  if (want < kInnerFloor) return inner_tol;  // no single round can finish
  return want < 0.1 ? want : 0.1;            // the loosest round that finishes
}

}  // namespace pdlp
