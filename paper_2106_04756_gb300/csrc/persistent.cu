// Persistent cooperative step kernel: the inner loop of Algorithm 1 (step
// attempts of Algorithm 2 between two evaluations, Section 3.1 / 3.4) in one
// launch of one 512-thread CTA per SM.
//
// Per attempt:
//   primal phase  x' = proj_X(x - tau (c - K^T y)) over the rows of K^T (eq. (3))
//   grid barrier
//   dual phase    y' = proj_Y(y + sigma (q - 2 K x' + K x)) over the rows of K
//   grid barrier  (after each CTA published its partial sums)
//   step test     every CTA sums all partials in the same fixed order and runs
//                 Algorithm 2's test on its own copy of the step control, so all
//                 CTAs take the same decision without a third barrier.
//
// Work placement: each warp of the grid owns a fixed list of warp chunks of
// K^T and of K for the whole launch (assign_chunks: a longest-processing-time
// assignment under a cost model of the chunks, so that the warps, and with
// them the SMs, reach the grid barriers together); the descriptors are
// copied into the warp's shared-memory slice once per launch.
// A warp keeps two chunks in flight: while one is reduced, the loads of the
// next (column indices, then values, row starts and epilogue operands by
// cp.async, and the gathered entries through L2) are outstanding.  The
// phases are bound by the rate of scattered gathers.  Per-row arithmetic is
// that of k_primal / k_dual; only the grouping of the three step-test sums
// differs.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <queue>
#include <vector>

#include "common.cuh"
#include "evaluate.cuh"
#include "solver.cuh"

namespace pdlp {

namespace {

constexpr int kPThreads = 512;
constexpr int kPWarps = kPThreads / 32;
constexpr int kMaxAttemptsPerLaunch = 4096;
__host__ __device__ inline int round16(int b) { return (b + 15) & ~15; }

// Asynchronous global -> shared copies (cp.async, cached in L1).  Used only
// for data no other CTA writes during the launch (matrix values, row starts
// and the warp's own rows' operands).  Entries written by other CTAs (the
// gathered vector) are plain loads when L1G: the grid barrier that precedes
// each phase then ends with an acquire of the arrival counter that every CTA
// released after its writes, so by the memory model the loads after it see
// those writes (an acquire at GPU scope discards stale L1 lines), and the
// gathers keep the L1 hits of rows that share columns.  That pays where the
// working set exceeds L2 (1M-node PageRank: 144 -> 112 us per float32
// attempt); where it stays in L2 the L2-only loads (ld.global.cg) without the
// acquire are faster (100k x 250k LP: 40.8 against 42.8 us in float64), so
// the choice is made per context (PersistGeo::l1_gather).
template <typename T>
__device__ __forceinline__ void cp_async(T *dst, const T *src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-warp staging buffer of one chunk in flight (buf_elems<PRE>() elements
// of T: values, gathered entries, row sums, then PRE epilogue operands per
// row; then kChunkRows + 1 ints of row starts).  A phase's PRE is its
// operands per row: 5 for the step phases.
constexpr int kPre = 5;
template <int PRE>
__host__ __device__ constexpr int buf_elems() {
  return 2 * kChunkNnz + kChunkRows + PRE * kChunkRows;
}
template <typename T, int PRE = kPre>
__host__ __device__ constexpr int buf_bytes() {
  return (int)((buf_elems<PRE>() * sizeof(T) + (kChunkRows + 1) * 4 + 15) / 16 * 16);
}

// Primal epilogue of eq. (3) for column j of K (row j of K^T).  Operands
// x_j, xs_j, c_j, l_j, u_j are staged (pre[k * 32 + lane]) with the chunk.
template <typename T>
struct PrimalPhase {
  const T *x, *xs, *cs, *ls, *us;
  T *xn, *xsn;
  T tau, et;
  static constexpr int NA = 1, PRE = kPre;
  double acc[NA];
  __device__ __forceinline__ void stage(int j, T *pre) const {
    cp_async(pre, x + j);
    cp_async(pre + 32, xs + j);
    cp_async(pre + 64, cs + j);
    cp_async(pre + 96, ls + j);
    cp_async(pre + 128, us + j);
  }
  __device__ __forceinline__ void load(int j, T *pre) const {
    pre[0] = __ldcg(x + j);
    pre[32] = __ldcg(xs + j);
    pre[64] = cs[j];
    pre[96] = ls[j];
    pre[128] = us[j];
  }
  __device__ __forceinline__ void epi(int j, T g, const T *pre, double *a) {
    const T xj = pre[0];
    const T xp = clampv<T>(xj - tau * (pre[64] - g), pre[96], pre[128]);
    xn[j] = xp;
    xsn[j] = pre[32] + et * xp;
    const T d = xp - xj;
    a[0] += (double)(d * d);
  }
};

// Dual epilogue of eq. (3) for row i of K, with the sums of Algorithm 2's
// test.  Staged operands: (Kx)_i, y_i, ys_i, q_i, ylo_i.
template <typename T>
struct DualPhase {
  const T *y, *Kx, *ys, *qs, *ylos;
  T *yn, *Kxn, *ysn;
  T sig, et;
  static constexpr int NA = 2, PRE = kPre;
  double acc[NA];
  __device__ __forceinline__ void stage(int i, T *pre) const {
    cp_async(pre, Kx + i);
    cp_async(pre + 32, y + i);
    cp_async(pre + 64, ys + i);
    cp_async(pre + 96, qs + i);
    cp_async(pre + 128, ylos + i);
  }
  __device__ __forceinline__ void load(int i, T *pre) const {
    pre[0] = __ldcg(Kx + i);
    pre[32] = __ldcg(y + i);
    pre[64] = __ldcg(ys + i);
    pre[96] = qs[i];
    pre[128] = ylos[i];
  }
  __device__ __forceinline__ void epi(int i, T kxn, const T *pre, double *a) {
    const T kx = pre[0], yi = pre[32], lo = pre[128];
    const T v = yi + sig * (pre[96] - T(2) * kxn + kx);
    const T yp = v > lo ? v : lo;
    yn[i] = yp;
    Kxn[i] = kxn;
    ysn[i] = pre[64] + et * yp;
    const T dy = yp - yi, dk = kxn - kx;
    a[0] += (double)(dy * dy);
    a[1] += (double)dy * (double)dk;
  }
};

// Copies the descriptors of the warp's chunks (its list of the balanced
// assignment) into shared memory; returns their count.
template <typename T>
__device__ int load_desc(const Mat<T> &A, int gw, Chunk *desc) {
  const int b = A.woff[gw], count = A.woff[gw + 1] - b;
  for (int i = threadIdx.x & 31; i < count; i += 32) desc[i] = A.chunks[A.wchunk[b + i]];
  __syncwarp();
  return count;
}

// Reduces a staged chunk and runs its epilogue: rows of a normal chunk by
// chunk_row_sums (the arithmetic of spmv_chunk), segments of long rows by
// a warp sum whose partials the last segment warp combines in segment order
// (that row's reduction terms go to its slot A.lr_acc).
template <typename T, typename Ph>
__device__ __forceinline__ void finish(const Mat<T> &A, const Chunk &c, char *buf, Ph &ph,
                                       const T (&xg)[kLaneItems]) {
  const int lane = threadIdx.x & 31;
  T *sval = reinterpret_cast<T *>(buf);
  T *sx = sval + kChunkNnz;
  T *srow = sx + kChunkNnz;
  T *pre = srow + kChunkRows;
  const int *srp = reinterpret_cast<const int *>(sval + buf_elems<Ph::PRE>());
  const int nb = c.nnz_begin, cnt = c.nnz_end - nb;
  if (c.row_end >= 0) {
    const int nrows = c.row_end - c.row_begin;
#pragma unroll
    for (int it = 0; it < kLaneItems; ++it) {
      const int e = lane + 32 * it;
      if (e < cnt) sx[stg<T>(e)] = xg[it];
    }
    __syncwarp();
    int s_r = 0, e_r = 0;
    if (lane < nrows) {
      s_r = srp[lane] - nb;
      e_r = lane + 1 < nrows ? srp[lane + 1] - nb : cnt;
    }
    chunk_row_sums<T, 1>(sval, sx, nrows, cnt, s_r, e_r, srow);
    __syncwarp();
    if (lane < nrows) ph.epi(c.row_begin + lane, srow[lane], pre + lane, ph.acc);
    return;
  }
  T acc = T(0);
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    if (e < cnt) acc = fma(sval[stg<T>(e)], xg[it], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lr = -(c.row_end + 1);
  const LongRow LR = A.longrows[lr];
  const int seg = (nb - __ldg(A.rp + LR.row)) / kSegNnz;
  int last = 0;
  if (lane == 0) {
    A.seg_part[LR.part_off + seg] = (double)acc;
    __threadfence();
    const unsigned prev = atomicAdd(A.seg_cnt + lr, 1u);
    last = prev == (unsigned)(LR.nseg - 1);
    if (last) A.seg_cnt[lr] = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  const double tot = warp_sum_parts(A.seg_part + LR.part_off, LR.nseg);
  if (lane == 0) {
    double la[Ph::NA];
#pragma unroll
    for (int a = 0; a < Ph::NA; ++a) la[a] = 0.0;
    ph.load(LR.row, pre);
    ph.epi(LR.row, (T)tot, pre, la);
#pragma unroll
    for (int a = 0; a < Ph::NA; ++a) A.lr_acc[(size_t)lr * kLrAcc + a] = la[a];
  }
}

// Starts the loads of one chunk: column indices (global, to registers), then
// values, row starts and epilogue operands by cp.async into the staging
// buffer `buf`, and the gathered vector entries into xg (through L1 when
// L1G, else through L2 only).
// issue() in two parts: issue_own starts every load but the gathers (data
// no other CTA writes during the phase before it: the matrix, the row
// starts, the warp's own rows' operands) and leaves the column indices in
// cj; issue_gather then loads the gathered entries.
template <typename T, typename Ph>
__device__ __forceinline__ void issue_own(const Mat<T> &A, const Chunk &c, const Ph &ph, char *buf,
                                          int (&cj)[kLaneItems]) {
  const int lane = threadIdx.x & 31;
  T *sval = reinterpret_cast<T *>(buf);
  T *pre = sval + 2 * kChunkNnz + kChunkRows;
  int *srp = reinterpret_cast<int *>(sval + buf_elems<Ph::PRE>());
  const int nb = c.nnz_begin, cnt = c.nnz_end - nb;
  const int nrows = c.row_end >= 0 ? c.row_end - c.row_begin : 0;
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    cj[it] = e < cnt ? __ldg(A.ci + nb + e) : 0;
    if (e < cnt) cp_async(sval + stg<T>(e), A.val + nb + e);
  }
  if (lane < nrows) {
    cp_async(srp + lane, A.rp + c.row_begin + lane);
    ph.stage(c.row_begin + lane, pre + lane);
  }
  cp_async_commit();
}

template <typename T, bool L1G>
__device__ __forceinline__ void issue_gather(const Chunk &c, const T *vec, const int (&cj)[kLaneItems],
                                             T (&xg)[kLaneItems]) {
  const int lane = threadIdx.x & 31;
  const int cnt = c.nnz_end - c.nnz_begin;
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    xg[it] = e < cnt ? (L1G ? vec[cj[it]] : __ldcg(vec + cj[it])) : T(0);
  }
}

// issue_own then issue_gather in one (kept as one body: the split form
// compiles to a slower float64 kernel, 162 -> 173 us per PageRank 1M attempt)
template <typename T, bool L1G, typename Ph>
__device__ __forceinline__ void issue(const Mat<T> &A, const Chunk &c, const T *vec, const Ph &ph, char *buf,
                                      T (&xg)[kLaneItems]) {
  const int lane = threadIdx.x & 31;
  T *sval = reinterpret_cast<T *>(buf);
  T *pre = sval + 2 * kChunkNnz + kChunkRows;
  int *srp = reinterpret_cast<int *>(sval + buf_elems<Ph::PRE>());
  const int nb = c.nnz_begin, cnt = c.nnz_end - nb;
  const int nrows = c.row_end >= 0 ? c.row_end - c.row_begin : 0;
  int cj[kLaneItems];
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    cj[it] = e < cnt ? __ldg(A.ci + nb + e) : 0;
    if (e < cnt) cp_async(sval + stg<T>(e), A.val + nb + e);
  }
  if (lane < nrows) {
    cp_async(srp + lane, A.rp + c.row_begin + lane);
    ph.stage(c.row_begin + lane, pre + lane);
  }
  cp_async_commit();
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    xg[it] = e < cnt ? (L1G ? vec[cj[it]] : __ldcg(vec + cj[it])) : T(0);
  }
}

// float64 form of the pre-barrier start: only the cp.async copies (values,
// row starts, operands) before the wait, nothing held in registers across
// it; issue_idx_gather then loads the column indices and the gathers.
template <typename T, typename Ph>
__device__ __forceinline__ void issue_copies(const Mat<T> &A, const Chunk &c, const Ph &ph, char *buf) {
  const int lane = threadIdx.x & 31;
  T *sval = reinterpret_cast<T *>(buf);
  T *pre = sval + 2 * kChunkNnz + kChunkRows;
  int *srp = reinterpret_cast<int *>(sval + buf_elems<Ph::PRE>());
  const int nb = c.nnz_begin, cnt = c.nnz_end - nb;
  const int nrows = c.row_end >= 0 ? c.row_end - c.row_begin : 0;
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    if (e < cnt) cp_async(sval + stg<T>(e), A.val + nb + e);
  }
  if (lane < nrows) {
    cp_async(srp + lane, A.rp + c.row_begin + lane);
    ph.stage(c.row_begin + lane, pre + lane);
  }
  cp_async_commit();
}

template <typename T, bool L1G>
__device__ __forceinline__ void issue_idx_gather(const Mat<T> &A, const Chunk &c, const T *vec,
                                                 T (&xg)[kLaneItems]) {
  const int lane = threadIdx.x & 31;
  const int nb = c.nnz_begin, cnt = c.nnz_end - nb;
  int cj[kLaneItems];
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    cj[it] = e < cnt ? __ldg(A.ci + nb + e) : 0;
  }
#pragma unroll
  for (int it = 0; it < kLaneItems; ++it) {
    const int e = lane + 32 * it;
    xg[it] = e < cnt ? (L1G ? vec[cj[it]] : __ldcg(vec + cj[it])) : T(0);
  }
}

// The first two chunks' issue_own before a grid wait (their column indices
// in cj0 / cj1); run_phase(..., pre = true) then only gathers for them.
template <typename T, typename Ph>
__device__ __forceinline__ void issue_first(const Mat<T> &A, const Chunk *desc, int count, const Ph &ph, char *wsm,
                                            int (&cj0)[kLaneItems], int (&cj1)[kLaneItems]) {
  if (count > 0) issue_own<T>(A, desc[0], ph, wsm, cj0);
  if (count > 1) issue_own<T>(A, desc[1], ph, wsm + buf_bytes<T, Ph::PRE>(), cj1);
}

// Fixed-order CTA sum of three values per thread with few float64 adds
// (float64 is slow on this part): value a's 512 terms go to the staging area
// of warp a (idle between the phases), which sums them, 16 per lane in a
// pairwise tree, then in a 5-step shuffle.  tot[0..2] (shared) holds the
// sums after the call.
static_assert(kPThreads * sizeof(double) <= 2 * buf_bytes<float>(), "a warp's staging area holds a CTA's terms");
__device__ __forceinline__ void cta_sum3(const double (&v)[3], char *sm, int warp_bytes, double *tot) {
  __syncthreads();  // every warp is done with its staging buffers
#pragma unroll
  for (int a = 0; a < 3; ++a) reinterpret_cast<double *>(sm + (size_t)a * warp_bytes)[threadIdx.x] = v[a];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 3) {
    const double *r = reinterpret_cast<const double *>(sm + (size_t)w * warp_bytes);
    double p[kPThreads / 32];
#pragma unroll
    for (int k = 0; k < kPThreads / 32; ++k) p[k] = r[lane + 32 * k];
#pragma unroll
    for (int s = kPThreads / 64; s >= 1; s >>= 1) {
#pragma unroll
      for (int k = 0; k < s; ++k) p[k] += p[k + s];
    }
    double t = p[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) tot[w] = t;
  }
  __syncthreads();
}

// One phase over the warp's chunks with two chunks in flight (two staging
// buffers, gathered entries in registers a / b): the loads of chunk i + 2
// start once chunk i is done.
template <typename T, bool L1G, typename Ph>
__device__ __forceinline__ void run_phase(const Mat<T> &A, const Chunk *desc, int count, const T *vec, char *wsm,
                                          Ph &ph, bool pre = false, const int (&cj0)[kLaneItems] = {},
                                          const int (&cj1)[kLaneItems] = {}) {
  char *b0 = wsm, *b1 = wsm + buf_bytes<T, Ph::PRE>();
  T ga[kLaneItems], gb[kLaneItems];
  if (sizeof(T) == 4 && pre) {
    if (count > 0) issue_gather<T, L1G>(desc[0], vec, cj0, ga);
    if (count > 1) issue_gather<T, L1G>(desc[1], vec, cj1, gb);
  } else if (pre) {
    if (count > 0) issue_idx_gather<T, L1G>(A, desc[0], vec, ga);
    if (count > 1) issue_idx_gather<T, L1G>(A, desc[1], vec, gb);
  } else {
    if (count > 0) issue<T, L1G>(A, desc[0], vec, ph, b0, ga);
    if (count > 1) issue<T, L1G>(A, desc[1], vec, ph, b1, gb);
  }
  for (int i = 0; i < count; i += 2) {
    if (i + 1 < count)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    __syncwarp();
    finish<T>(A, desc[i], b0, ph, ga);
    __syncwarp();
    if (i + 2 < count) issue<T, L1G>(A, desc[i + 2], vec, ph, b0, ga);
    if (i + 1 < count) {
      if (i + 2 < count)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
      __syncwarp();
      finish<T>(A, desc[i + 1], b1, ph, gb);
      __syncwarp();
      if (i + 3 < count) issue<T, L1G>(A, desc[i + 3], vec, ph, b1, gb);
    }
  }
}

// A phase whose product A v the persistent evaluation just stored (prod):
// the epilogues of the warp's chunks in the same order as run_phase, on the
// stored sums (bit-identical to the gathered ones: the same chunk lists and
// row sums), without the gathers; a long row's epilogue once, by the warp of
// its first segment.
template <typename T, typename Ph>
__device__ __forceinline__ void reuse_phase(const Mat<T> &A, const Chunk *desc, int count, const T *prod,
                                            char *wsm, Ph &ph) {
  const int lane = threadIdx.x & 31;
  T *pre = reinterpret_cast<T *>(wsm) + 2 * kChunkNnz + kChunkRows;
  for (int i = 0; i < count; ++i) {
    const Chunk c = desc[i];
    if (c.row_end >= 0) {
      const int nrows = c.row_end - c.row_begin;
      if (lane < nrows) {
        const int j = c.row_begin + lane;
        ph.load(j, pre + lane);
        ph.epi(j, __ldcg(prod + j), pre + lane, ph.acc);
      }
    } else if (lane == 0) {
      const int lr = -(c.row_end + 1);
      const LongRow LR = A.longrows[lr];
      if (c.nnz_begin == __ldg(A.rp + LR.row)) {
        double la[Ph::NA];
#pragma unroll
        for (int a = 0; a < Ph::NA; ++a) la[a] = 0.0;
        ph.load(LR.row, pre);
        ph.epi(LR.row, __ldcg(prod + LR.row), pre, la);
#pragma unroll
        for (int a = 0; a < Ph::NA; ++a) A.lr_acc[(size_t)lr * kLrAcc + a] = la[a];
      }
    }
    __syncwarp();
  }
}

template <typename T, bool L1G>
__global__ void __launch_bounds__(kPThreads, 1)
    k_persist(Mat<T> K, Mat<T> KT, Problem<T> P, State<T> S, PersistGeo geo) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double s_tot[3];
  __shared__ double fac[2][kMaxEval];
  __shared__ StepCtl ctl;
  __shared__ long long s_fac_k0, s_iter_limit, s_attempt_limit;
  __shared__ int s_eval_every;
  __shared__ unsigned long long s_base, s_wait_ns;
  __shared__ int s_wait_extra, s_reuse;
  Scalars *sc = S.s;
  const int wid = threadIdx.x >> 5;
  const int gw = blockIdx.x * kPWarps + wid;
  const unsigned long long G = gridDim.x;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(S.tickets + kTicketBar);
  char *wsm = sm + (size_t)geo.warp_bytes * wid;
  Chunk *dp = reinterpret_cast<Chunk *>(wsm + geo.o_desc_p);
  Chunk *dd = reinterpret_cast<Chunk *>(wsm + geo.o_desc_d);
  if (threadIdx.x == 0) {
    load_step(sc, ctl);
    s_fac_k0 = sc->fac_k0;
    s_iter_limit = sc->iter_limit;
    s_attempt_limit = sc->attempt_limit;
    s_eval_every = sc->eval_every;
    s_wait_ns = sc->wait_ns;
    s_wait_extra = sc->wait_extra;
    s_reuse = sc->kty_valid;  // K^T y of the current y stored by the persistent evaluation
    // the counter is a multiple of G between launches; CTAs that already
    // arrived at the first barrier add less than G
    const unsigned long long c0 = *reinterpret_cast<volatile unsigned long long *>(bar);
    s_base = c0 / G * G;
  }
  const int ne = sc->eval_every < kMaxEval ? sc->eval_every : kMaxEval;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    fac[0][i] = sc->fac_tab[0][i];
    fac[1][i] = sc->fac_tab[1][i];
  }
  const int cnt_p = load_desc(KT, gw, dp);
  const int cnt_d = load_desc(K, gw, dd);
  __syncthreads();
  unsigned long long target = s_base;
  for (int att = 0; att < kMaxAttemptsPerLaunch; ++att) {
    if (ctl.status != kRunning || ctl.chunk_acc >= s_eval_every || ctl.k >= s_iter_limit ||
        ctl.attempts >= s_attempt_limit)
      break;
    const int cur = ctl.cur;
    PrimalPhase<T> pp{S.x[cur], S.xs[cur], P.cs, P.ls, P.us, S.x[cur ^ 1], S.xs[cur ^ 1],
                      (T)ctl.tau, (T)ctl.eta, {0.0}};
    if (att == 0 && s_reuse)
      reuse_phase<T>(KT, dp, cnt_p, S.KTy_cur, wsm, pp);
    else
      run_phase<T, L1G>(KT, dp, cnt_p, S.y[cur], wsm, pp);
    target += G + (att == 0 && s_wait_extra ? 1ull : 0ull);
    // arrive, start the dual phase's first two chunks (data no other CTA
    // writes in the primal phase, which writes only x' and its running sum),
    // then wait for the other CTAs.  float32 also loads their column indices
    // before the wait (100k x 250k LP float32 attempt 30.9 -> 29.9 us,
    // PageRank 1M unchanged at 112 us); float64 only the copies, since its
    // indices held across the wait spill (PageRank 1M 162.1 -> 179.8 us)
    grid_arrive(bar);
    DualPhase<T> dph{S.y[cur], S.Kx[cur], S.ys[cur], P.qs, P.ylos, S.y[cur ^ 1], S.Kx[cur ^ 1], S.ys[cur ^ 1],
                     (T)ctl.sigma, (T)ctl.eta, {0.0, 0.0}};
    if constexpr (sizeof(T) == 4) {
      int cj0[kLaneItems], cj1[kLaneItems];
      issue_first<T>(K, dd, cnt_d, dph, wsm, cj0, cj1);
      if (!grid_wait(bar, target, &sc->err, s_wait_ns, L1G)) {
        cp_async_wait<0>();  // the copies in flight land before the kernel returns
        break;
      }
      run_phase<T, L1G>(K, dd, cnt_d, S.x[cur ^ 1], wsm, dph, true, cj0, cj1);
    } else {
      if (cnt_d > 0) issue_copies<T>(K, dd[0], dph, wsm);
      if (cnt_d > 1) issue_copies<T>(K, dd[1], dph, wsm + buf_bytes<T, DualPhase<T>::PRE>());
      if (!grid_wait(bar, target, &sc->err, s_wait_ns, L1G)) {
        cp_async_wait<0>();  // the copies in flight land before the kernel returns
        break;
      }
      run_phase<T, L1G>(K, dd, cnt_d, S.x[cur ^ 1], wsm, dph, true);
    }
    {
      const double v[3] = {pp.acc[0], dph.acc[0], dph.acc[1]};
      cta_sum3(v, sm, geo.warp_bytes, s_tot);
      if (threadIdx.x == 0) {
        S.part_cp[3 * blockIdx.x + 0] = s_tot[0];
        S.part_cp[3 * blockIdx.x + 1] = s_tot[1];
        S.part_cp[3 * blockIdx.x + 2] = s_tot[2];
      }
    }
    target += G;
    if (!grid_barrier(bar, target, &sc->err, s_wait_ns, L1G)) break;
    {
      // the same fixed-order sum in every CTA, all loads in one round: each
      // thread adds its per-CTA partials, then its rows split into segments
      double t[3] = {0.0, 0.0, 0.0};
      for (int b = threadIdx.x; b < (int)G; b += blockDim.x) {
        t[0] += __ldcg(S.part_cp + 3 * b + 0);
        t[1] += __ldcg(S.part_cp + 3 * b + 1);
        t[2] += __ldcg(S.part_cp + 3 * b + 2);
      }
      for (int r = threadIdx.x; r < KT.nlong; r += blockDim.x) t[0] += __ldcg(KT.lr_acc + (size_t)r * kLrAcc);
      for (int r = threadIdx.x; r < K.nlong; r += blockDim.x) {
        t[1] += __ldcg(K.lr_acc + (size_t)r * kLrAcc);
        t[2] += __ldcg(K.lr_acc + (size_t)r * kLrAcc + 1);
      }
      cta_sum3(t, sm, geo.warp_bytes, s_tot);
      if (threadIdx.x == 0) {
        t[0] = s_tot[0];
        t[1] = s_tot[1];
        t[2] = s_tot[2];
        const long long idx = ctl.k - s_fac_k0;
        double fr, fg;
        if (idx >= 0 && idx < ne) {
          fr = fac[0][idx];
          fg = fac[1][idx];
        } else {
          const double kk = (double)(ctl.k + 1);
          fr = 1.0 - pow(kk + 1.0, -0.3);
          fg = 1.0 + pow(kk + 1.0, -0.6);
        }
        const long long k_before = ctl.k;
        const double eta_try = ctl.eta;
        step_update(ctl, t[0], t[1], t[2], fr, fg);
        if (S.eta_log && blockIdx.x == 0 && ctl.k > k_before) S.eta_log[k_before] = eta_try;
      }
      __syncthreads();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    store_step(sc, ctl);
    sc->kty_valid = 0;  // y moved (or the stored product was used)
  }
}

// ------------------------------------------------ persistent evaluation
//
// The products and Eq. (15) terms of an evaluation in one launch of one
// 512-thread CTA per SM, on the step kernel's balanced chunk lists, with two
// chunks in flight per warp (separate evaluation kernels ran in 1.6 and 1.15
// waves of CTAs, with idle SMs in their tails):
//   A  K^T y  (current iterate): (K~^T y)_j stored, column terms of candidate 0
//   B  K^T ys (average, when there is one): (K~^T ys)_j stored, candidate 1
//   C  K xs   (average): (K~ xs)_i stored, row terms of both candidates
// The phases share no data, so no grid barrier separates them; B uses its
// own long-row segment partials, arrival counters and epilogue slots (4..7)
// (the matrix KTb), so that a warp in B never meets a warp still in A on a
// long row.  Per-CTA sums go to S.part_ce; the last CTA adds them and the
// long-row slots in a fixed order and finishes the evaluation.  The
// epilogue arithmetic is that of k_eval_cols / k_eval_rows.  Float64 only:
// the operands are staged with the chunk as float64.
constexpr int kEvalPre = 8;

// Column terms for candidate c (scale 1: the current iterate; 1 / sum_eta:
// the average, from its running sums): [c^T x, ||rc - lambda||^2,
// l^T lambda+ - u^T lambda-, ||x - x0||^2 (scaled)].
struct ColEvalPhase {
  const double *xv, *x0, *c, *l, *u, *D2, *D2inv;
  double *prod;
  double scale;
  static constexpr int NA = 4, PRE = kEvalPre;
  double acc[NA];
  __device__ __forceinline__ void stage(int j, double *pre) const {
    cp_async(pre, xv + j);
    cp_async(pre + 32, x0 + j);
    cp_async(pre + 64, c + j);
    cp_async(pre + 96, l + j);
    cp_async(pre + 128, u + j);
    cp_async(pre + 160, D2 + j);
    cp_async(pre + 192, D2inv + j);
  }
  __device__ __forceinline__ void load(int j, double *pre) const {
    pre[0] = __ldcg(xv + j);
    pre[32] = __ldcg(x0 + j);
    pre[64] = c[j];
    pre[96] = l[j];
    pre[128] = u[j];
    pre[160] = D2[j];
    pre[192] = D2inv[j];
  }
  __device__ __forceinline__ void epi(int j, double g, const double *pre, double *a) {
    prod[j] = g;
    const double xt = pre[0] * scale, kt = g * scale;  // (exact for scale 1)
    const double xr = pre[32], cj = pre[64], lj = pre[96], uj = pre[128], D2j = pre[160], iD2 = pre[192];
    const bool lf = !d_is_neginf(lj), uf = !d_is_posinf(uj);
    const double xo = D2j * xt, rc = cj - kt * iD2;
    const bool lam_rc = lf ? (uf || d_gt0(rc)) : (uf && d_lt0(rc));
    const double lam = lam_rc ? rc : 0.0;
    const double d = lam_rc ? (d_finite(rc) ? 0.0 : __longlong_as_double(0x7ff8000000000000ll)) : rc;
    a[0] += cj * xo;
    a[1] = fma(d, d, a[1]);
    if (d_gt0(lam) || d_lt0(lam)) a[2] = __dadd_rn(a[2], __dmul_rn(d_gt0(lam) ? lj : uj, lam));
    a[3] += (xt - xr) * (xt - xr);
  }
};

// Row terms of both candidates: [||(q - K x)+||^2, q^T y, ||y - y0||^2
// (scaled), general dual bound term] for the current iterate, then the
// average.
struct RowEvalPhase {
  const double *y, *ys, *Kx, *y0, *q, *D1, *D1inv, *ylo;
  double *Kxbar;
  double inv;
  bool avg;
  static constexpr int NA = 8, PRE = kEvalPre;
  double acc[NA];
  __device__ __forceinline__ void stage(int i, double *pre) const {
    cp_async(pre, y + i);
    cp_async(pre + 32, ys + i);
    cp_async(pre + 64, Kx + i);
    cp_async(pre + 96, y0 + i);
    cp_async(pre + 128, q + i);
    cp_async(pre + 160, D1 + i);
    cp_async(pre + 192, D1inv + i);
    cp_async(pre + 224, ylo + i);
  }
  __device__ __forceinline__ void load(int i, double *pre) const {
    pre[0] = __ldcg(y + i);
    pre[32] = __ldcg(ys + i);
    pre[64] = __ldcg(Kx + i);
    pre[96] = __ldcg(y0 + i);
    pre[128] = q[i];
    pre[160] = D1[i];
    pre[192] = D1inv[i];
    pre[224] = ylo[i];
  }
  __device__ __forceinline__ void epi(int i, double s, const double *pre, double *a) {
    Kxbar[i] = s;
    const double yr = pre[96], qi = pre[128], D1i = pre[160], iD1 = pre[192], lo = pre[224];
    const bool ineq = !d_is_neginf(lo), lo_nz = d_gt0(lo) || d_lt0(lo);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 1 && !avg) break;
      const double yt = c == 0 ? pre[0] : pre[32] * inv;
      const double kx = c == 0 ? pre[64] : s * inv;
      double r = qi - kx * iD1;
      if (ineq) {
        if (lo_nz) a[4 * c + 3] += lo * r;
        r = d_gt0(r) ? r : 0.0;
      }
      a[4 * c + 0] += r * r;
      a[4 * c + 1] += qi * (D1i * yt);
      a[4 * c + 2] += (yt - yr) * (yt - yr);
    }
  }
};

// Terms t0 and t0 + 1 (of 16) summed over `nb` CTA partials (stride 16) and
// terms l0, l0 + 1 of the long-row slots `lr` ([nlong][kLrAcc]), by one
// warp, valid in lane 0; every load before any sum.
__device__ __forceinline__ void pe_terms2(const double *part, int nb, int t0, const double *lr, int nlong, int l0,
                                          double (&out)[2]) {
  const int lane = threadIdx.x & 31;
  double acc[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[q][u] = 0.0;
  for (int b0 = lane; b0 < nb; b0 += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + 32 * u;
      if (b < nb) {
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q][u] += __ldcg(part + (size_t)b * 16 + t0 + q);
      }
    }
  }
  for (int r0 = lane; r0 < nlong; r0 += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 32 * u;
      if (r < nlong) {
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q][u] += __ldcg(lr + (size_t)r * kLrAcc + l0 + q);
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

template <bool L1G>
__global__ void __launch_bounds__(kPThreads, 1)
    k_eval_persist(Mat<double> K, Mat<double> KT, Mat<double> KTb, Problem<double> P, State<double> S,
                   PersistGeo geo) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double ecr[16];
  Scalars *sc = S.s;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kPWarps + wid;
  char *wsm = sm + (size_t)geo.warp_bytes * wid;
  Chunk *dp = reinterpret_cast<Chunk *>(wsm + geo.o_desc_p);
  Chunk *dd = reinterpret_cast<Chunk *>(wsm + geo.o_desc_d);
  const int cur = sc->cur;
  const bool avg = sc->sum_eta > 0.0;
  const double inv = avg ? 1.0 / sc->sum_eta : 0.0;
  {
    // Algorithm 2's factors for the next chunk's steps (k does not change
    // until then): entry i by lane 0 of the last warp of CTA i mod grid
    const long long k0 = sc->k;
    const int ne = sc->eval_every < kMaxEval ? sc->eval_every : kMaxEval;
    if (wid == kPWarps - 1 && lane == 0) {
      for (int i = blockIdx.x; i < ne; i += gridDim.x) {
        const double kk = (double)(k0 + i + 1);
        sc->fac_tab[0][i] = 1.0 - pow(kk + 1.0, -0.3);
        sc->fac_tab[1][i] = 1.0 + pow(kk + 1.0, -0.6);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->fac_k0 = k0;
  }
  const int cnt_p = load_desc(KT, gw, dp);
  const int cnt_d = load_desc(K, gw, dd);
  ColEvalPhase pa{S.x[cur], S.x0, P.c, P.l, P.u, P.D2, P.D2inv, S.KTy_cur, 1.0, {0.0, 0.0, 0.0, 0.0}};
  run_phase<double, L1G>(KT, dp, cnt_p, S.y[cur], wsm, pa);
  ColEvalPhase pb{S.xs[cur], S.x0, P.c, P.l, P.u, P.D2, P.D2inv, S.KTys, inv, {0.0, 0.0, 0.0, 0.0}};
  if (avg) run_phase<double, L1G>(KTb, dp, cnt_p, S.ys[cur], wsm, pb);
  RowEvalPhase pc{S.y[cur], S.ys[cur], S.Kx[cur], S.y0, P.q, P.D1, P.D1inv, P.ylo, S.Kxbar, inv, avg, {}};
#pragma unroll
  for (int a = 0; a < 8; ++a) pc.acc[a] = 0.0;
  run_phase<double, L1G>(K, dd, cnt_d, S.xs[cur], wsm, pc);
  // fixed-order CTA sums of the 16 terms: term a's 512 values go to area a
  // of the (now idle) staging space, which warp a adds
  double v[16];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = pa.acc[a];
    v[4 + a] = pb.acc[a];
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) v[8 + a] = pc.acc[a];
  __syncthreads();
  double *red = reinterpret_cast<double *>(sm);
#pragma unroll
  for (int a = 0; a < 16; ++a) red[a * kPThreads + threadIdx.x] = v[a];
  __syncthreads();
  {
    const double *r = red + wid * kPThreads;
    double p[kPThreads / 32];
#pragma unroll
    for (int k = 0; k < kPThreads / 32; ++k) p[k] = r[lane + 32 * k];
#pragma unroll
    for (int s = kPThreads / 64; s >= 1; s >>= 1) {
#pragma unroll
      for (int k = 0; k < s; ++k) p[k] += p[k + s];
    }
    double t = p[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) S.part_ce[(size_t)blockIdx.x * 16 + wid] = t;
  }
  if (!last_block(S.tickets + kTicketMisc)) return;
  // warp w < 8: terms 2w, 2w + 1 (columns: slots of KT's long rows, phase B
  // in slots 4..7; rows: slots of K's long rows)
  if (wid < 8) {
    double t2[2];
    if (wid < 4) pe_terms2(S.part_ce, gridDim.x, 2 * wid, KT.lr_acc, KT.nlong, 2 * wid, t2);
    else pe_terms2(S.part_ce, gridDim.x, 2 * wid, K.lr_acc, K.nlong, 2 * wid - 8, t2);
    if (lane == 0) {
      ecr[2 * wid] = t2[0];
      ecr[2 * wid + 1] = t2[1];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sc->kty_valid = 1;  // phase A's K^T y serves the next chunk's first step
  eval_finish(sc, ecr, S.trace);
}

// Reopens a finished state for timing: running status, no limits, a zero
// barrier counter and the step factors of the next steps.
__global__ void k_persist_reopen(Scalars *s, unsigned *tickets) {
  if (threadIdx.x == 0) {
    s->chunk_acc = 0;
    s->status = kRunning;
    s->err = 0;
    s->iter_limit = 1ll << 62;
    s->attempt_limit = 1ll << 62;
    s->fac_k0 = s->k;
    s->kty_valid = 0;  // timed attempts gather K^T y
    tickets[kTicketBar] = 0u;
    tickets[kTicketBar + 1] = 0u;
  }
  __syncthreads();
  fill_step_factors(s);
}

template <typename T>
void layout(PersistGeo &g, int cmax_p, int cmax_d) {
  g.o_desc_p = 2 * buf_bytes<T>();
  g.o_desc_d = g.o_desc_p + 16 * cmax_p;
  g.warp_bytes = round16(g.o_desc_d + 16 * cmax_d);
  g.smem = g.warp_bytes * kPWarps;
}

}  // namespace

int persist_warps_per_cta() { return kPWarps; }

int persist_warps() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms * kPWarps;
}

template <typename T>
cudaError_t persist_plan(int cmax_kt, int cmax_k, int assign_nw, int mode, int l1_gather, PersistGeo *pg) {
  *pg = PersistGeo{};
  if (mode == 0) return cudaSuccess;
  cudaError_t e;
  int dev = 0, sms = 0, optin = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, k_persist<T, true>))) return e;
  const int budget = optin - (int)fa.sharedSizeBytes;
  const int grid = sms;
  if (grid * kPWarps != assign_nw) return cudaSuccess;  // no assignment for this grid
  PersistGeo g{};
  g.grid = grid;
  g.l1_gather = l1_gather;
  layout<T>(g, cmax_kt, cmax_k);
  if (g.smem > budget) return cudaSuccess;  // too many chunks per warp: one launch per half-step
  // the attribute is per kernel, shared by every context: set it to the budget
  if ((e = cudaFuncSetAttribute(k_persist<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget))) return e;
  if ((e = cudaFuncSetAttribute(k_persist<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget))) return e;
  int per = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist<T, true>, kPThreads, g.smem))) return e;
  if (per < 1) return cudaSuccess;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist<T, false>, kPThreads, g.smem))) return e;
  if (per < 1) return cudaSuccess;
  *pg = g;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_persist(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                           const PersistGeo &pg, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)pg.grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = (size_t)pg.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (pg.l1_gather) return cudaLaunchKernelEx(&cfg, k_persist<T, true>, K, KT, P, S, pg);
  return cudaLaunchKernelEx(&cfg, k_persist<T, false>, K, KT, P, S, pg);
}

// Layout of the persistent evaluation kernel on the step kernel's grid and
// chunk lists (8 staged operands per row); pe->grid = 0 (the separate
// evaluation kernels run instead) for float32 or when it does not fit.
template <typename T>
cudaError_t eval_plan(const PersistGeo &pg, int cmax_kt, int cmax_k, PersistGeo *pe) {
  *pe = PersistGeo{};
  if constexpr (sizeof(T) != 8) {
    return cudaSuccess;
  } else {
    if (pg.grid <= 0) return cudaSuccess;
    cudaError_t e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_eval_persist<true>))) return e;
    const int budget = optin - (int)fa.sharedSizeBytes;
    PersistGeo g{};
    g.grid = pg.grid;
    g.l1_gather = pg.l1_gather;
    g.o_desc_p = 2 * buf_bytes<double, kEvalPre>();
    g.o_desc_d = g.o_desc_p + 16 * cmax_kt;
    g.warp_bytes = round16(g.o_desc_d + 16 * cmax_k);
    g.smem = g.warp_bytes * kPWarps;
    // the CTA sums reuse the staging space: 16 terms x kPThreads doubles
    if (g.smem > budget || g.smem < 16 * kPThreads * (int)sizeof(double)) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(k_eval_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget))) return e;
    if ((e = cudaFuncSetAttribute(k_eval_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget))) return e;
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eval_persist<true>, kPThreads, g.smem))) return e;
    if (per < 1) return cudaSuccess;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eval_persist<false>, kPThreads, g.smem))) return e;
    if (per < 1) return cudaSuccess;
    *pe = g;
    return cudaSuccess;
  }
}

// One evaluation by the persistent evaluation kernel (float64 contexts with
// pe.grid > 0).  KTb is KT with the second set of long-row buffers.
template <typename T>
cudaError_t launch_eval_persist(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                                const State<T> &S, const PersistGeo &pe, cudaStream_t st) {
  if constexpr (sizeof(T) != 8) {
    return cudaErrorNotSupported;
  } else {
    if (pe.grid <= 0) return cudaErrorInvalidValue;
    if (pe.l1_gather)
      k_eval_persist<true><<<pe.grid, kPThreads, pe.smem, st>>>(K, KT, KTb, P, S, pe);
    else
      k_eval_persist<false><<<pe.grid, kPThreads, pe.smem, st>>>(K, KT, KTb, P, S, pe);
    return cudaGetLastError();
  }
}

// Mean duration of one launch of the persistent evaluation kernel, event-timed
// over `reps` launches on `st` after one untimed launch (each evaluates the
// state as it stands; 0 when the context has no such kernel).
template <typename T>
cudaError_t time_eval_persist(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                              const State<T> &S, const PersistGeo &pe, int reps, cudaStream_t st, float *ms) {
  *ms = 0.f;
  if (pe.grid <= 0) return cudaSuccess;
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0))) return e;
  if ((e = cudaEventCreate(&e1))) {
    cudaEventDestroy(e0);
    return e;
  }
  e = launch_eval_persist<T>(K, KT, KTb, P, S, pe, st);
  if (!e) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && !e; ++r) e = launch_eval_persist<T>(K, KT, KTb, P, S, pe, st);
  if (!e) e = cudaEventRecord(e1, st);
  if (!e) e = cudaEventSynchronize(e1);
  float a = 0.f;
  if (!e) e = cudaEventElapsedTime(&a, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!e) *ms = a / (float)reps;
  return e;
}

// Mean duration of one step attempt inside the persistent kernel: `reps`
// launches (each runs until eval_every steps are accepted), event-timed on
// `st`, divided by the attempts they made.
template <typename T>
cudaError_t time_persist(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                         const PersistGeo &pg, int reps, cudaStream_t st, float *ms_attempt) {
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0))) return e;
  if ((e = cudaEventCreate(&e1))) {
    cudaEventDestroy(e0);
    return e;
  }
  Scalars h0, h1;
  double total = 0.0;
  long long att = 0;
  for (int r = 0; r < reps && !e; ++r) {
    k_persist_reopen<<<1, 64, 0, st>>>(S.s, S.tickets);
    if ((e = cudaMemcpyAsync(&h0, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st))) break;
    cudaEventRecord(e0, st);
    e = launch_persist<T>(K, KT, P, S, pg, st);
    cudaEventRecord(e1, st);
    if (!e) e = cudaMemcpyAsync(&h1, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) break;
    float a = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    total += a;
    att += h1.attempts - h0.attempts;
    if (h1.status != kRunning || h1.err) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_attempt = att > 0 ? (float)(total / att) : 0.f;
  return e;
}

#define PDLP_INST(T)                                                                                        \
  template cudaError_t persist_plan<T>(int, int, int, int, int, PersistGeo *);                                   \
  template cudaError_t launch_persist<T>(const Mat<T> &, const Mat<T> &, const Problem<T> &, const State<T> &, \
                                         const PersistGeo &, cudaStream_t);                                 \
  template cudaError_t time_persist<T>(const Mat<T> &, const Mat<T> &, const Problem<T> &, const State<T> &,   \
                                       const PersistGeo &, int, cudaStream_t, float *);                                      \
  template cudaError_t eval_plan<T>(const PersistGeo &, int, int, PersistGeo *);                                  \
  template cudaError_t time_eval_persist<T>(const Mat<T> &, const Mat<T> &, const Mat<T> &, const Problem<T> &,   \
                                            const State<T> &, const PersistGeo &, int, cudaStream_t, float *); \
  template cudaError_t launch_eval_persist<T>(const Mat<T> &, const Mat<T> &, const Mat<T> &, const Problem<T> &, \
                                              const State<T> &, const PersistGeo &, cudaStream_t);
PDLP_INST(double)
PDLP_INST(float)
#undef PDLP_INST

}  // namespace pdlp
