// Slab step kernels: the two half-steps of one step attempt (Eq. (3) with
// Algorithm 2's reductions) over fixed-size slabs of kSlabNnz nonzeros, one
// warp per slab, for LPs whose working set exceeds L2.
//
// Why slabs: on GB300 the sparse products of large LPs are bound by the
// L1TEX unit's rate for scattered gathers, so the kernel must keep every SM
// full of independent gathers and spend few other instructions per nonzero.
// A slab gives each warp the same number of nonzeros whatever the row
// lengths (power-law rows, a dense row), lets each lane load its eight
// consecutive column indices and values with 128-bit loads, and needs about
// 32 registers per thread, so 64 warps per SM stay resident.  Each launch
// only reads the vector it gathers (written by the previous launch), so the
// gathers go through the L1-cached read-only path.
//
// Per slab (lane l owns nonzeros 8l .. 8l+7):
//   products v_k * vec[col_k] in registers;
//   row starts of the slab's rows as a 256-bit mask in shared memory;
//   a lane-local pass adds the products by row; a segmented inclusive scan
//   over the lanes (5 steps) completes rows that cross lanes; each complete
//   row's sum lands in srow[its start position];
//   the epilogue runs one lane per row of the slab (coalesced operands);
//   a row that crosses into the next slab and ends there is finished by the
//   slab holding its start, which reads the remaining nonzeros itself (the
//   next slab skips them); rows reaching further (split rows) get one
//   partial per slab, and the last slab warp to finish adds them in slab
//   order and runs that row's epilogue, whose reduction terms go to the
//   row's own slot.
// Every sum has a fixed order, so results are bitwise reproducible.
#pragma once

#include "common.cuh"

namespace pdlp {

constexpr int kSlabThreads = 256;
constexpr int kSlabWarps = kSlabThreads / 32;
static_assert(kSlabNnz == 32 * 8, "eight nonzeros per lane");

__host__ __device__ inline int slab_ctas(int nslab) { return (nslab + kSlabWarps - 1) / kSlabWarps; }

// First slab of this CTA's contiguous range (of CTA blockIdx.x + next) when
// nslab slabs are split evenly over the grid.
__device__ __forceinline__ int slab_begin(int nslab, int next = 0) {
  return (int)(((long long)(blockIdx.x + next) * nslab) / gridDim.x);
}

template <typename T>
struct Load8;
template <>
struct Load8<float> {
  static __device__ __forceinline__ void run(const float *p, float (&o)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
};
template <>
struct Load8<double> {
  static __device__ __forceinline__ void run(const double *p, double (&o)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + i);
      o[2 * i] = a.x;
      o[2 * i + 1] = a.y;
    }
  }
};
__device__ __forceinline__ void load8i(const int32_t *p, int (&o)[8]) {
  const int4 a = __ldg(reinterpret_cast<const int4 *>(p)), b = __ldg(reinterpret_cast<const int4 *>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

// A split row over more than kSlabDeferSlabs slabs (a dense row) is
// deferred: its slabs only store their partials, and the launch's last CTA
// adds them and runs the row's epilogue (finish_deferred), so that thousands
// of slabs do not each fence and count on one counter at the end of the
// launch.
constexpr int kSlabDeferSlabs = 32;
__host__ __device__ inline bool split_deferred(const SplitRow &R) { return R.s_last - R.s_first + 1 > kSlabDeferSlabs; }

// One slab's partial of split row `id` (whole warp): lane 0 stores it and
// counts the arrival; the last of the row's slabs adds all partials in slab
// order (lanes strided, then a fixed shuffle tree) and lane 0 runs the row's
// epilogue into the row's slot of split_acc.
template <typename T, int NA, typename Epi>
__device__ __forceinline__ void split_arrive(const Mat<T> &A, int id, int s, double part, Epi &epi) {
  const int lane = threadIdx.x & 31;
  const SplitRow R = A.splits[id];
  if (split_deferred(R)) {
    if (lane == 0) A.split_part[R.part_off + (s - R.s_first)] = part;
    return;
  }
  int last = 0;
  if (lane == 0) {
    A.split_part[R.part_off + (s - R.s_first)] = part;
    __threadfence();
    const unsigned prev = atomicAdd(A.split_cnt + id, 1u);
    last = prev == (unsigned)(R.s_last - R.s_first);
    if (last) A.split_cnt[id] = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  const double tot = warp_sum_parts(A.split_part + R.part_off, R.s_last - R.s_first + 1);
  if (lane == 0) {
    double la[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) la[a] = 0.0;
    epi(R.row, (T)tot, la);
#pragma unroll
    for (int a = 0; a < NA; ++a) A.split_acc[(size_t)id * kLrAcc + a] = la[a];
  }
}

// Row sums of slab s of A against the gathered vector `vec` and the epilogue
// epi(row, sum, acc) of every row the slab completes (whole warp).  `bits`
// (8 words) and `srow` (kSlabNnz entries) are the warp's shared memory.
template <typename T, int NA, typename Epi>
__device__ __forceinline__ void slab_warp(const Mat<T> &A, int s, const T *__restrict__ vec, unsigned *bits, T *srow,
                                          double (&acc)[NA], Epi &epi) {
  const int lane = threadIdx.x & 31;
  const int base = s * kSlabNnz;
  const int e0 = base + 8 * lane;
  int col[8];
  T v[8], g[8];
  load8i(A.ci + e0, col);
  Load8<T>::run(A.val + e0, v);
#pragma unroll
  for (int k = 0; k < 8; ++k) g[k] = __ldg(vec + col[k]);
  if (lane < 8) bits[lane] = 0u;
  __syncwarp();
  const int fr = __ldg(A.slab_first + s), fr1 = __ldg(A.slab_first + s + 1);
  for (int r = fr + lane; r < fr1; r += 32) {
    const int b = __ldg(A.rp + r), e = __ldg(A.rp + r + 1);
    if (e > b) atomicOr(bits + ((b - base) >> 5), 1u << ((b - base) & 31));
  }
  __syncwarp();
  const unsigned b8 = (bits[lane >> 2] >> (8 * (lane & 3))) & 0xffu;
  // lane-local pass: runs of consecutive nonzeros of one row
  T run = T(0), headv = T(0);
  bool started = false;
  int spos = -1;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((b8 >> k) & 1u) {
      if (!started) headv = run;  // the run continuing an earlier lane's row
      else srow[spos] = run;      // a row that starts and ends in this lane
      started = true;
      spos = 8 * lane + k;
      run = T(0);
    }
    run = fma(v[k], g[k], run);
  }
  // segmented inclusive scan of the lanes' last runs: a chain restarts at a
  // lane holding a row start; sp carries the start position of the chain
  T sv = run;
  int f = started ? 1 : 0, sp = started ? spos : -1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T tv = __shfl_up_sync(0xffffffffu, sv, d);
    const int tf = __shfl_up_sync(0xffffffffu, f, d);
    const int tp = __shfl_up_sync(0xffffffffu, sp, d);
    if (lane >= d) {
      if (!f) {
        sv = tv + sv;
        sp = tp;
      }
      f |= tf;
    }
  }
  T pv = __shfl_up_sync(0xffffffffu, sv, 1);
  int pp = __shfl_up_sync(0xffffffffu, sp, 1);
  if (lane == 0) {
    pv = T(0);
    pp = -1;
  }
  // the chain that ends just before this lane's first start
  T head_part = T(0);
  bool head_here = false;
  if (started) {
    if (pp >= 0) srow[pp] = pv + headv;
    else if (lane > 0 || !(b8 & 1u)) {  // the slab's head run
      head_part = pv + headv;
      head_here = true;
    }
  }
  const int hs = __ldg(A.slab_head + s), ts = __ldg(A.slab_tail + s);
  // the chain that reaches the slab's end
  if (lane == 31) {
    if (sp < 0) {  // no row starts in the slab: all of it is the head run
      head_part = sv;
      head_here = true;
    } else if (ts == -1) {
      srow[sp] = sv;
    }
  }
  if (ts <= kSlabExtend) {
    // the last row ends in the next slab: read its remainder here (at most
    // kSlabNnz nonzeros, lanes strided, fixed shuffle tree)
    const int er = __ldg(A.rp + (kSlabExtend - ts) + 1);
    T ext = T(0);
    for (int k = base + kSlabNnz + lane; k < er; k += 32) ext = fma(__ldg(A.val + k), __ldg(vec + __ldg(A.ci + k)), ext);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ext += __shfl_xor_sync(0xffffffffu, ext, o);
    if (lane == 31) srow[sp] = sv + ext;
  }
  __syncwarp();
  for (int r = fr + lane; r < fr1; r += 32) {
    const int b = __ldg(A.rp + r), e = __ldg(A.rp + r + 1);
    if (e - base > kSlabNnz && ts >= 0) continue;  // reaches past the next slab: a split row
    const T sum = e > b ? srow[b - base] : T(0);
    epi(r, sum, acc);
  }
  if (hs >= 0) {
    const unsigned hm = __ballot_sync(0xffffffffu, head_here);
    const T hv = __shfl_sync(0xffffffffu, head_part, hm ? __ffs(hm) - 1 : 0);
    split_arrive<T, NA>(A, hs, s, (double)hv, epi);
  }
  if (ts >= 0) {
    const T tv = __shfl_sync(0xffffffffu, sv, 31);
    split_arrive<T, NA>(A, ts, s, (double)tv, epi);
  }
}

// The deferred split rows of A (whole CTA, after every slab of the launch
// stored its partials): per row, each warp adds a contiguous eighth of the
// partials, thread 0 adds the warps' sums in order and runs the row's
// epilogue into its slot of split_acc.  `sh` holds kSlabWarps doubles.
template <typename T, int NA, typename Epi>
__device__ __forceinline__ void finish_deferred(const Mat<T> &A, Epi &epi, double *sh) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int id = 0; id < A.nsplit; ++id) {
    const SplitRow R = A.splits[id];
    if (!split_deferred(R)) continue;
    const int np = R.s_last - R.s_first + 1;
    const int b = (int)((long long)wid * np / kSlabWarps), e = (int)((long long)(wid + 1) * np / kSlabWarps);
    const double ws = warp_sum_parts(A.split_part + R.part_off + b, e - b);
    if (lane == 0) sh[wid] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < kSlabWarps; ++w) tot += sh[w];
      double la[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) la[a] = 0.0;
      epi(R.row, (T)tot, la);
#pragma unroll
      for (int a = 0; a < NA; ++a) A.split_acc[(size_t)id * kLrAcc + a] = la[a];
    }
    __syncthreads();
  }
}

// Fixed-order sum of the NA epilogue sums of A's split rows; result valid in
// thread 0.
template <int NA, typename M>
__device__ __forceinline__ void sum_split_rows(const M &A, double (&out)[NA], double *red) {
#pragma unroll
  for (int a = 0; a < NA; ++a) out[a] = 0.0;
  for (int r = threadIdx.x; r < A.nsplit; r += blockDim.x) {
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] += __ldcg(A.split_acc + (size_t)r * kLrAcc + a);
  }
  block_sum<NA>(out, red);
}

}  // namespace pdlp
