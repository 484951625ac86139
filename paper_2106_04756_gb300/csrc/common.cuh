// Internal definitions shared by the library's translation units.
//
// Layout in device memory (one context = one LP):
//   K   CSR: row_ptr int32[m+1], col_idx int32[nnz], values T[nnz]
//   K^T CSR: built on the device by a stable radix sort of K's entries by column
//   vectors: contiguous arrays of T (float64 or float32) per quantity
//   scalars: one `Scalars` block (float64 / int64) read by every kernel
// Sparse products use a CSR-stream scheme at warp granularity: rows are
// grouped into warp chunks of at most kChunkNnz nonzeros and kChunkRows rows;
// each warp stages its chunk's values and gathered vector entries in its own
// shared-memory slice with coalesced loads, reduces each row with a
// power-of-two group of lanes and runs the fused epilogue one lane per row.
// Rows longer than kSegNnz are split into segments of kSegNnz nonzeros whose
// partial sums are combined, in segment order, by the last segment warp to
// finish.  All reductions are deterministic: fixed thread-to-data assignment
// and fixed combination order.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pdlp.h"
#include "schedule.h"

namespace pdlp {

constexpr int kThreads = 256;          // CTA size of the sparse-product kernels
constexpr int kWarps = kThreads / 32;  // warps per CTA, one chunk per warp
constexpr int kGapBuckets = 2048;      // radix digit of the normalized-gap selection
constexpr int kGapThreads = 512;
constexpr int kGapSlots = 3;           // current, average, restart point
constexpr int kMaxEval = 256;          // largest eval_every (step-factor table size)
constexpr int kLrAcc = 8;              // epilogue sums kept per long row
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // default bound of a grid-barrier wait

// CSR matrix plus its warp-chunk schedule.
template <typename T>
struct Mat {
  int32_t rows, cols;
  const int32_t *rp, *ci;
  const T *val;
  const Chunk *chunks;
  int32_t nchunks;
  int32_t nblocks;        // CTAs = ceil(nchunks / kWarps)
  const LongRow *longrows;
  double *seg_part;       // one partial per long-row segment (per gathered vector)
  unsigned int *seg_cnt;  // arrival counter per long row
  double *lr_acc;         // epilogue sums of each long row [nlong][kLrAcc]
  int32_t nlong;
  // chunks of each warp of the persistent kernel: wchunk[woff[w] .. woff[w+1])
  // for its assign_nw warps (a cost-balanced static assignment)
  const int32_t *wchunk = nullptr, *woff = nullptr;
  int32_t assign_nw = 0;
  // fixed-size slabs of kSlabNnz nonzeros (build_slabs; the index and value
  // arrays are zero-padded to nslab * kSlabNnz entries).  slab_on: the step
  // attempts of this precision run on the slab kernels.
  int32_t nslab = 0, nsplit = 0, slab_on = 0;
  int32_t ndefer = 0;                   // split rows over more than kSlabDeferSlabs slabs
  int32_t slab_grid = 0;                // CTAs of a slab launch (at most the resident count)
  const int32_t *slab_first = nullptr;  // [nslab + 1]
  const int32_t *slab_head = nullptr, *slab_tail = nullptr;  // [nslab]
  const SplitRow *splits = nullptr;     // [nsplit]
  double *split_part = nullptr;         // one partial per (split row, slab)
  unsigned int *split_cnt = nullptr;    // arrival counter per split row
  double *split_acc = nullptr;          // epilogue sums of each split row [nsplit][kLrAcc]
};

// Solver outcome codes (same values as the public PDLP_* status codes).
enum : int { kRunning = 0, kOptimal = 1, kIterLimit = 2, kKktLimit = 3, kTimeLimit = 4, kNumErr = 5,
             kWaitTimeout = 6, kStalled = 9 };  // kStalled: refinement inner solves only

// Every scalar of Algorithm 1 / 2 / 3 and of the evaluation, in one block.
struct Scalars {
  // --- Algorithm 2 step control
  double eta;       // step size of the next attempt
  double omega;     // primal weight omega^n
  double tau, sigma;  // eta / omega and eta * omega of the next attempt (Section 2)
  double inv_omega;   // 1 / omega
  // Algorithm 2 factors 1 - (k+1)^-0.3 and 1 + (k+1)^-0.6 for the steps
  // k = fac_k0 + i of the current chunk (k counted from 1), filled by block 0
  // of each evaluation's row kernel (k_eval_rows) and by fill_step_factors
  double fac_tab[2][kMaxEval];
  long long fac_k0;
  double sum_eta;   // sum of accepted step sizes of this outer loop
  double dx2, dy2, inter, eta_bar;  // reductions of the last attempt
  // --- restart state (Section 3.2)
  double mu0;       // mu_n(z^{n,0}, z^{n-1,0}); +inf in the first outer loop
  double muc_prev;  // candidate mu of the previous evaluation in this outer loop
  double inv_avg;   // 1 / sum_eta at the evaluation
  double mu[kGapSlots];
  double gval[kGapSlots];
  // --- evaluation (Eq. (15) on the original problem), [candidate][term]
  double kkt[2][8];
  double cand_dx2[2], cand_dy2[2];  // squared distances to z^{n,0} (scaled space)
  double pw_omega[2], pw_inv[2], pw_r2[2];  // Algorithm 3 per candidate (primal weight, 1/it, slot-2 radius^2)
  double qnorm, cnorm;              // ||q||_2, ||c||_2 of the original problem
  double rel_tol;
  // --- gap radix selection per slot
  double g_r2[kGapSlots], g_omega[kGapSlots], g_inv_omega[kGapSlots];
  double g_W[kGapSlots], g_V[kGapSlots], g_A[kGapSlots];
  unsigned int g_prefix[kGapSlots];
  int g_active[kGapSlots];
  // --- options
  double beta_suff, beta_nec, beta_art, pw_theta, eps_zero;
  // --- counters and flags
  long long k, t, attempts, restarts;
  long long iter_limit, attempt_limit;
  unsigned long long t0_ns, time_limit_ns, t_end_ns;
  int cur;        // which of the two buffers holds the current iterate
  int kty_valid;  // KTy_cur holds K^T y of the current y, from the persistent evaluation
  int chunk_acc;  // accepted iterations since the last evaluation
  int eval_every;
  int status;
  int ret_which;  // 0 current, 1 average
  int phase;      // 0 before the first step, 1 in the loop
  int do_gap;     // this evaluation runs the restart test
  int restart;    // a restart was decided at this evaluation
  int cand;       // restart candidate: 0 current, 1 average
  int adaptive_restart, pw_update;
  int err;        // bounded-wait failures (device-side timeouts)
  int const_step; // 1: constant step size (every attempt accepted)
  int trace_n;    // restart evaluations recorded so far (ring of kTraceCap)
  // --- Appendix C.2 restart variants
  int restart_to_current;  // 0: the restart candidate is always the average
  int vrestart;            // no-restart mode: primal weight updated at this evaluation
  long long k_virt;        // no-restart mode: k of the last primal weight update
  // --- Appendix C.1 Malitsky-Pock line search (mp = 1)
  int mp;
  int mp_trial;            // trials of the current iteration so far
  double mp_eta_k, mp_theta;  // eta_k and theta_k = eta_{k-1} / eta_k of the current iterate
  double mp_eh, mp_th;        // candidate eta_hat and theta_hat of the next trial
  double mp_bf, mp_df, mp_ic; // breaking, downscaling, interpolation
  // --- stall test of refinement inner solves (stall_evals > 0)
  double stall_best;          // smallest relative Eq. (15) error at an evaluation so far
  int stall_count, stall_evals;
  // --- bounded device waits
  unsigned long long wait_ns; // bound of each grid-barrier wait
  int wait_extra;             // 1: the first barrier of each persistent launch waits for
                              // one arrival more than the grid has (timeout-path test)
};

// One record per restart evaluation: k, t, mu_cur, mu_avg, mu0, candidate,
// restart (0/1), omega after the update, then the radii r_cur, r_avg, and
// the relative Eq. (15) terms (gap, primal, dual) of the current and the
// average iterate.
constexpr int kTraceCap = 2048;
constexpr int kTraceLen = 16;

// An LP in the form of Eq. (1) on the device: preconditioned data (type T,
// read in the iteration) and original-space data (float64, read by the
// termination test).
template <typename T>
struct Problem {
  int32_t m, n;
  const T *cs, *qs, *ls, *us, *ylos;
  const double *c, *q, *l, *u, *ylo;  // ylo: 0 / -inf for the paper's Y, general for corrections
  const double *D1, *D2;
  const double *D1inv, *D2inv;  // 1 / D1, 1 / D2 (the evaluation multiplies instead of dividing)
};

// Iteration state (ping-pong buffers selected by Scalars::cur).
template <typename T>
struct State {
  T *x[2], *y[2], *Kx[2], *xs[2], *ys[2];
  T *x0, *y0;                  // restart point z^{n,0}
  T *KTy_cur, *KTys, *Kxbar;   // products at the evaluation
  double *part_p, *part_d;     // per-CTA partials of the primal / dual kernels
  double *part_cp;             // per-CTA partials of the persistent kernel [CTA][3]
  double *part_sp, *part_sd;   // per-CTA partials of the slab step kernels (primal [CTA], dual [CTA][2])
  double *part_ec, *part_er;   // per-CTA partials of the evaluation kernels
  double *part_ce;             // per-CTA partials of the persistent evaluation kernel [CTA][16]
  unsigned int *tickets;       // arrival counters (one per kernel kind)
  unsigned int *gtickets;      // arrival counters of the evaluation CTA groups (columns, then rows)
  Scalars *s;
  unsigned int *gkeys;         // gap keys [kGapSlots][n + m]
  double *ghist;               // gap histogram [kGapSlots][3][kGapBuckets] (w, v, a)
  unsigned int *gmask;         // nonempty buckets of the gap histogram [kGapSlots][kGapBuckets / 32]
  double *xo, *yo;             // returned point (original space, float64)
  double *trace;               // [kTraceCap][kTraceLen]
  double *eta_log;             // nullable: step size of each accepted step, by step index
};

// Arrival counters; [kTicketBar, kTicketBar + 1] hold the 64-bit barrier
// counter of the persistent kernel (8-byte aligned).
enum TicketId { kTicketDual = 0, kTicketEvalRows = 1, kTicketGap = 2, kTicketMisc = 3, kTicketBar = 4,
                kTicketSlabPrimal = 6, kNumTickets = 8 };

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Comparisons of a float64 with zero and infinity by tests on its bits,
// with the results of the float64 comparisons for every input (signed
// zeros, infinities, NaN): a float64 comparison holds a sub-partition's
// float64 unit for tens of cycles on this part, an integer test does not.
__device__ __forceinline__ bool d_gt0(double v) {  // v > 0
  const long long b = __double_as_longlong(v);
  return b > 0ll && b <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool d_lt0(double v) {  // v < 0
  const long long b = __double_as_longlong(v), m = b & 0x7fffffffffffffffll;
  return b < 0ll && m != 0ll && m <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool d_finite(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool d_is_neginf(double v) { return __double_as_longlong(v) == (long long)0xfff0000000000000ull; }
__device__ __forceinline__ bool d_is_posinf(double v) { return __double_as_longlong(v) == 0x7ff0000000000000ll; }

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Deterministic sum of NV per-thread values over the CTA; the result is
// valid in thread 0.  `red` must hold NV * (blockDim.x / 32) doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * nw + warp] = v[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = lane < nw ? red[a * nw + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[a] = t;
    }
  }
}

// Deterministic CTA sum of NV per-thread values with few float64 instructions
// (float64 throughput is low on this part): values go to shared memory, one
// warp adds blockDim/32 of them per lane, then a 5-step shuffle.  The result
// is valid in thread 0.  `red` must hold NV * blockDim.x doubles.
template <int NV>
__device__ __forceinline__ void block_sum_lean(double (&v)[NV], double *red) {
  const int nt = blockDim.x, lane = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) red[a * nt + threadIdx.x] = v[a];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = 0.0;
      for (int k = lane; k < nt; k += 32) t += red[a * nt + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[a] = t;
    }
  }
}

// Fixed-order sum of np partials p[0], p[stride], ... by one warp, with
// eight independent loads in flight per lane (a row split into thousands of
// segments would otherwise leave one warp waiting on a long chain of
// dependent loads at the end of a phase); the total is valid in lane 0.
__device__ __forceinline__ double warp_sum_parts(const double *p, int np, int stride = 1) {
  const int lane = threadIdx.x & 31;
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = 0.0;
  for (int b = 0; b < np; b += 256) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = b + 32 * u + lane;
      if (k < np) a[u] += __ldcg(p + (size_t)k * stride);
    }
  }
  double t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  return t;
}

// Fixed-order sum of `count` partials (stride `stride`, offset `off`) by one
// CTA; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void sum_partials(const double *part, int count, int stride,
                                             double (&out)[NV], double *red) {
  // four independent accumulators per thread keep four loads in flight
  double acc[4][NV];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[u][a] = 0.0;
  }
  const int nt = blockDim.x;
  for (int b0 = threadIdx.x; b0 < count; b0 += 4 * nt) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * nt;
      if (b < count) {
#pragma unroll
        for (int a = 0; a < NV; ++a) acc[u][a] += __ldcg(part + (size_t)b * stride + a);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = (acc[0][a] + acc[1][a]) + (acc[2][a] + acc[3][a]);
  block_sum<NV>(out, red);
}

// Fixed-order sum of the NA epilogue sums of A's long rows (after their
// producers finished); result valid in thread 0.
template <int NA, typename M>
__device__ __forceinline__ void sum_long_rows(const M &A, double (&out)[NA], double *red) {
#pragma unroll
  for (int a = 0; a < NA; ++a) out[a] = 0.0;
  for (int r = threadIdx.x; r < A.nlong; r += blockDim.x) {
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] += __ldcg(A.lr_acc + (size_t)r * kLrAcc + a);
  }
  block_sum<NA>(out, red);
}

// True in every thread of the CTA that arrives last at `ticket`; that CTA
// also resets the ticket.  Writes made before the call are visible to it.
__device__ __forceinline__ bool last_block(unsigned int *ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(ticket, 1u);
    s_last = (prev == gridDim.x - 1);
    if (s_last) *ticket = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// last_block over several launches sharing `ticket`: true in the CTA that
// arrives last among `total` CTAs (which may belong to kernels running
// concurrently); that CTA resets the ticket.
__device__ __forceinline__ bool last_of(unsigned int *ticket, unsigned int total) {
  __shared__ int s_last_of;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(ticket, 1u);
    s_last_of = (prev == total - 1u);
    if (s_last_of) *ticket = 0u;
  }
  __syncthreads();
  if (s_last_of) __threadfence();
  return s_last_of != 0;
}

// ------------------------------------------------------- CSR-stream engine
//
// spmv_warp computes, for the calling warp's chunk of `A`, the row sums
// sum_k A_ik * v_a[col_k] for NV gathered vectors v_a and calls
// epi(row, sums, acc) once per row: lane r for row r of a chunk (coalesced),
// or lane 0 for a long row.  `acc` is where the epilogue adds its NA
// reduction terms: the caller's per-thread array, except for rows split into
// segments, whose terms go to the row's own slot A.lr_acc[row][0..NA) (the
// warp that runs that epilogue depends on timing; consumers add the slots in
// row order after the per-CTA partials).  Warps work independently:
//   staging: each lane loads up to kChunkNnz/32 column indices and values
//            (coalesced, independent), then the gathered entries, into the
//            warp's shared-memory slice;
//   rows:    a power-of-two group of L lanes per row (L * rows <= 32) sums the
//            row from shared memory, then shuffles; rows longer than a
//            threshold the chunk picks from its row lengths are summed by the
//            whole warp instead (chunk_row_sums);
//   segments of rows longer than kSegNnz: warp partials combined, in segment
//            order, by the last segment warp to arrive.
// All sums have a fixed order (deterministic).  `wsm` is the warp's slice of
// spmv_warp_smem<T>(NV) bytes.
constexpr int kLaneItems = kChunkNnz / 32;
constexpr unsigned kSegSteps = kSegStepsHost;  // float64 steps above which a chunk takes the segmented row sums

// Position of a chunk's nonzero e in its staging arrays.  In float64 the
// 16-byte granules (two entries) of each aligned group of eight are permuted
// by an XOR with e / 8 mod 8, so that lanes reading eight consecutive entries
// each (chunk_row_sums_seg) fall on different banks; the permutation stays
// inside each 128-byte group, so lanes writing consecutive entries stay
// conflict-free too.  float32: identity.
template <typename T>
__device__ __forceinline__ int stg(int e) {
  if constexpr (sizeof(T) == 8) return (((e >> 1) ^ ((e >> 3) & 7)) << 1) | (e & 1);
  else return e;
}

// Position of the n-th (n >= 1) set bit of m.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  int pos = 0;
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) {
    const int c = __popc(m & ((1u << sh) - 1u));
    if (n > c) {
      n -= c;
      m >>= sh;
      pos += sh;
    }
  }
  return pos;
}

// Segmented row sums of a float64 chunk (one gathered vector): lane l
// multiplies its eight consecutive nonzeros [8l, 8l + 8) and adds them by
// row; a row that crosses lane boundaries is completed by an inclusive
// segmented scan over the lanes (5 steps) of each lane's last partial sum.
// 8 multiply-adds and about 6 adds per lane, whatever the row lengths.  Row
// r's sum goes to srow[r] (0 for an empty row).  Fixed order throughout.
template <typename T>
__device__ __forceinline__ void chunk_row_sums_seg(const T *sval, const T *sx, int nrows, int cnt, int s_r,
                                                   int e_r, T *srow) {
  const int lane = threadIdx.x & 31;
  const bool mine = lane < nrows;
  const bool nonempty_row = mine && e_r > s_r;
  const unsigned nonempty = __ballot_sync(0xffffffffu, nonempty_row);
  if (mine && !nonempty_row) srow[lane] = T(0);
  // bit p of starts[p / 32]: a non-empty row starts at local position p
  unsigned starts[kChunkNnz / 32];
#pragma unroll
  for (int w = 0; w < kChunkNnz / 32; ++w)
    starts[w] = __reduce_or_sync(0xffffffffu, (nonempty_row && (s_r >> 5) == w) ? (1u << (s_r & 31)) : 0u);
  const int e0 = 8 * lane;
  const int nloc = cnt - e0 < 0 ? 0 : (cnt - e0 < 8 ? cnt - e0 : 8);
  // row of item e0: the rank-th non-empty row, rank = starts at or before e0
  int rank = 0;
#pragma unroll
  for (int w = 0; w < kChunkNnz / 32; ++w) {
    if (e0 >= 32 * w + 32) rank += __popc(starts[w]);
    else if (e0 >= 32 * w) rank += __popc(starts[w] & (0xffffffffu >> (31 - (e0 - 32 * w))));
  }
  // the word holding this lane's eight items and the next lane's first item
  // (selected without dynamic indexing, so that starts[] stays in registers)
  const int w0 = e0 >> 5, en = e0 + 8, w1 = en >> 5;
  unsigned word = 0u, word_n = 0u;
#pragma unroll
  for (int w = 0; w < kChunkNnz / 32; ++w) {
    if (w == w0) word = starts[w];
    if (w == w1) word_n = starts[w];
  }
  const bool first_is_start = nloc > 0 && ((word >> (e0 & 31)) & 1u);
  int cur = rank > 0 ? nth_set_bit(nonempty, rank) : 0;
  const int head_row = cur;
  T acc = T(0), headv = T(0);
  bool crossed = false;  // a row start after e0 inside this lane
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    if (it < nloc) {
      const int e = e0 + it;
      if (it > 0 && ((word >> (e & 31)) & 1u)) {
        if (!crossed && !first_is_start) headv = acc;  // continuation of an earlier lane's row
        else srow[cur] = acc;                          // a row that starts and ends in this lane
        crossed = true;
        const int nxt = __ffs(cur < 31 ? nonempty & ~((2u << cur) - 1u) : 0u) - 1;  // next non-empty row
        cur = nxt >= 0 ? nxt : cur;
        acc = T(0);
      }
      acc = fma(sval[stg<T>(e)], sx[stg<T>(e)], acc);
    }
  }
  // carries of the rows that cross lanes: segmented inclusive scan of the
  // lanes' last partial sums; a chain starts at a lane whose last partial
  // begins at a row start
  T v = acc;
  int f = (nloc == 0 || crossed || first_is_start) ? 1 : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T tv = __shfl_up_sync(0xffffffffu, v, d);
    const int tf = __shfl_up_sync(0xffffffffu, f, d);
    if (lane >= d) {
      if (!f) v = tv + v;
      f = f | tf;
    }
  }
  const T carry_prev = __shfl_up_sync(0xffffffffu, v, 1);
  if (nloc > 0 && !first_is_start && crossed) srow[head_row] = carry_prev + headv;
  // the last partial's row ends with this lane: the chunk ends, or the next
  // lane's first item starts a row
  const bool next_starts = en < cnt && ((word_n >> (en & 31)) & 1u);
  if (nloc > 0 && (e0 + nloc == cnt || next_starts)) srow[cur] = v;
}

// Row sums of one staged chunk of nrows <= 32 rows: values sval[stg(e)] and
// gathered entries sx[a * kChunkNnz + stg(e)] for the chunk's nonzeros e;
// lane r passes its row's local bounds [s_r, e_r) (any values on lanes >=
// nrows) and cnt is the chunk's nonzero count.
// Rows are summed by power-of-two groups of L lanes (L * nrows <= 32), which
// costs the warp ceil(max length / L) steps; with power-law row lengths one
// long row would set that count for the whole chunk, so rows longer than a
// threshold T are instead summed by the whole warp, one after another
// (ceil(length / 32) steps and a 5-step shuffle each).  T in {16, 32, 64,
// 128} or none is chosen per chunk by that integer step count; in float64
// with one vector, chunks whose step count stays above the segmented sum's
// (chunk_row_sums_seg, 8 + 6) take that instead.  Every sum has a fixed
// order.  Writes srow[a * kChunkRows + r].
template <typename T, int NV>
__device__ __forceinline__ void chunk_row_sums(const T *sval, const T *sx, int nrows, int cnt, int s_r, int e_r,
                                               T *srow) {
  const int lane = threadIdx.x & 31;
  int L = 32;
  while (L > 1 && L * nrows > 32) L >>= 1;
  const int lg = 31 - __clz(L);
  const bool mine = lane < nrows;
  const unsigned len = mine ? (unsigned)(e_r - s_r) : 0u;
  unsigned best = __reduce_max_sync(0xffffffffu, (len + (unsigned)L - 1u) >> lg);
  unsigned thr = 0xffffffffu;
#pragma unroll
  for (unsigned th = 16; th <= 128; th <<= 1) {
    const bool lng = len > th;
    const unsigned ms = __reduce_max_sync(0xffffffffu, lng ? 0u : (len + (unsigned)L - 1u) >> lg);
    const unsigned lc = __reduce_add_sync(0xffffffffu, lng ? ((len + 31u) >> 5) + 5u : 0u);
    if (ms + lc < best) {
      best = ms + lc;
      thr = th;
    }
  }
  if constexpr (sizeof(T) == 8 && NV == 1) {
    if (best + (unsigned)lg > kSegSteps) {
      chunk_row_sums_seg<T>(sval, sx, nrows, cnt, s_r, e_r, srow);
      return;
    }
  }
  // rows up to thr: groups of L lanes
  const int g = lane >> lg, gl = lane & (L - 1);
  const int gs = __shfl_sync(0xffffffffu, s_r, g), ge = __shfl_sync(0xffffffffu, e_r, g);
  const bool short_row = g < nrows && (unsigned)(ge - gs) <= thr;
  T acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = T(0);
  if (short_row) {
    for (int k = gs + gl; k < ge; k += L) {
      const int q = stg<T>(k);
      const T vv = sval[q];
#pragma unroll
      for (int a = 0; a < NV; ++a) acc[a] = fma(vv, sx[a * kChunkNnz + q], acc[a]);
    }
  }
  for (int o = L / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] += __shfl_down_sync(0xffffffffu, acc[a], o, L);
  }
  if (short_row && gl == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) srow[a * kChunkRows + g] = acc[a];
  }
  // longer rows: the whole warp, in row order
  unsigned lmask = __ballot_sync(0xffffffffu, mine && len > thr);
  while (lmask) {
    const int r = __ffs(lmask) - 1;
    lmask &= lmask - 1u;
    const int rs = __shfl_sync(0xffffffffu, s_r, r), re = __shfl_sync(0xffffffffu, e_r, r);
    T w[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) w[a] = T(0);
    for (int k = rs + lane; k < re; k += 32) {
      const int q = stg<T>(k);
      const T vv = sval[q];
#pragma unroll
      for (int a = 0; a < NV; ++a) w[a] = fma(vv, sx[a * kChunkNnz + q], w[a]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int a = 0; a < NV; ++a) w[a] += __shfl_down_sync(0xffffffffu, w[a], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) srow[a * kChunkRows + r] = w[a];
    }
  }
}

template <typename T>
__host__ __device__ constexpr size_t spmv_warp_smem(int nv) {
  return (size_t)kChunkNnz * sizeof(T) * (1 + nv) + (size_t)kChunkRows * sizeof(T) * nv;
}

template <typename T>
__host__ __device__ constexpr size_t spmv_smem_bytes(int nv) {
  return spmv_warp_smem<T>(nv) * kWarps;
}

// Loads of data other CTAs of the same launch may have written: through L2
// only when CG (L1 is not coherent across SMs), plain otherwise.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <typename T, int NV, int NA, bool CG = false, typename Epi>
__device__ __forceinline__ void spmv_chunk(const Mat<T> &A, int chunk, const T *const (&vec)[NV], char *wsm,
                                           double (&acc_out)[NA], Epi &&epi) {
  const int lane = threadIdx.x & 31;
  T *sval = reinterpret_cast<T *>(wsm);
  T *sx = sval + kChunkNnz;
  T *srow = sx + NV * kChunkNnz;
  const Chunk c = A.chunks[chunk];
  const int nb = c.nnz_begin, cnt = c.nnz_end - c.nnz_begin;
  if (c.row_end >= 0 && cnt <= kChunkNnz) {
    {
      int cj[kLaneItems];
      T v[kLaneItems];
#pragma unroll
      for (int it = 0; it < kLaneItems; ++it) {
        const int e = lane + 32 * it;
        cj[it] = e < cnt ? __ldg(A.ci + nb + e) : 0;
        v[it] = e < cnt ? __ldg(A.val + nb + e) : T(0);
      }
      T xv[NV][kLaneItems];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
#pragma unroll
        for (int it = 0; it < kLaneItems; ++it) {
          const int e = lane + 32 * it;
          xv[a][it] = e < cnt ? ldv<CG>(vec[a] + cj[it]) : T(0);
        }
      }
#pragma unroll
      for (int it = 0; it < kLaneItems; ++it) {
        const int e = lane + 32 * it;
        if (e < cnt) {
          const int q = stg<T>(e);
          sval[q] = v[it];
#pragma unroll
          for (int a = 0; a < NV; ++a) sx[a * kChunkNnz + q] = xv[a][it];
        }
      }
    }
    __syncwarp();
    const int nrows = c.row_end - c.row_begin;
    int s_r = 0, e_r = 0;
    if (lane < nrows) {
      s_r = __ldg(A.rp + c.row_begin + lane) - nb;
      e_r = __ldg(A.rp + c.row_begin + lane + 1) - nb;
    }
    chunk_row_sums<T, NV>(sval, sx, nrows, cnt, s_r, e_r, srow);
    __syncwarp();
    if (lane < nrows) {
      T s2[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) s2[a] = srow[a * kChunkRows + lane];
      epi(c.row_begin + lane, s2, acc_out);
    }
    return;
  }
  // a long row or a segment of one: the warp loops, kChunkNnz nonzeros per round
  T acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = T(0);
  for (int base = 0; base < cnt; base += kChunkNnz) {
    int cj[kLaneItems];
    T v[kLaneItems];
#pragma unroll
    for (int it = 0; it < kLaneItems; ++it) {
      const int e = base + lane + 32 * it;
      cj[it] = e < cnt ? __ldg(A.ci + nb + e) : 0;
      v[it] = e < cnt ? __ldg(A.val + nb + e) : T(0);
    }
#pragma unroll
    for (int it = 0; it < kLaneItems; ++it) {
      const int e = base + lane + 32 * it;
      if (e < cnt) {
#pragma unroll
        for (int a = 0; a < NV; ++a) acc[a] = fma(v[it], ldv<CG>(vec[a] + cj[it]), acc[a]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] += __shfl_down_sync(0xffffffffu, acc[a], o);
  }
  if (c.row_end >= 0) {
    if (lane == 0) epi(c.row_begin, acc, acc_out);
    return;
  }
  const int lr = -(c.row_end + 1);
  const LongRow L = A.longrows[lr];
  const int seg = (nb - __ldg(A.rp + L.row)) / kSegNnz;
  int last = 0;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) A.seg_part[(size_t)(L.part_off + seg) * NV + a] = (double)acc[a];
    __threadfence();
    const unsigned prev = atomicAdd(A.seg_cnt + lr, 1u);
    last = prev == (unsigned)(L.nseg - 1);
    if (last) A.seg_cnt[lr] = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  double tot[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) tot[a] = warp_sum_parts(A.seg_part + (size_t)L.part_off * NV + a, L.nseg, NV);
  if (lane == 0) {
    T t2[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) t2[a] = (T)tot[a];
    // the row's epilogue sums go to its own slot, summed in row order by the
    // consumer, so the result does not depend on which warp finished last
    double la[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) la[a] = 0.0;
    epi(L.row, t2, la);
#pragma unroll
    for (int a = 0; a < NA; ++a) A.lr_acc[(size_t)lr * kLrAcc + a] = la[a];
  }
}

// One chunk per warp, chunk index from the CTA and warp position.
template <typename T, int NV, int NA, typename Epi>
__device__ __forceinline__ void spmv_warp(const Mat<T> &A, const T *const (&vec)[NV], char *sm_cta,
                                          double (&acc)[NA], Epi &&epi) {
  const int wid = threadIdx.x >> 5;
  const int chunk = blockIdx.x * kWarps + wid;
  if (chunk >= A.nchunks) return;
  spmv_chunk<T, NV, NA, false>(A, chunk, vec, sm_cta + spmv_warp_smem<T>(NV) * wid, acc, epi);
}

// Grid-wide barrier of a cooperative launch on a monotonic 64-bit arrival
// counter: the n-th barrier of a launch whose counter started at `base`
// completes when the counter reaches base + n * gridDim.x.  The wait is
// bounded by limit_ns of %globaltimer (kBarrierTimeoutNs unless the options
// say otherwise): on expiry (or when another CTA has already failed) it
// records the failure in *err and returns false.
// grid_arrive + grid_wait: a CTA's arrival (after all its threads' writes),
// and the wait for the others; work between the two may read only data that
// no other CTA writes before its arrival.
__device__ __forceinline__ void grid_arrive(unsigned long long *count) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1ull);
  }
}

__device__ __forceinline__ bool grid_wait(unsigned long long *count, unsigned long long target, int *err,
                                          unsigned long long limit_ns, bool acquire = true) {
  __shared__ int s_okw;
  if (threadIdx.x == 0) {
    volatile unsigned long long *vc = count;
    volatile int *verr = err;
    int ok = 1;
    if (*vc < target) {
      const unsigned long long t0 = global_timer_ns();
      unsigned spins = 0;
      while (*vc < target) {
        if ((++spins & 63u) == 0u && (*verr || global_timer_ns() - t0 > limit_ns)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(8);
      }
    }
    if (ok && acquire) {
      unsigned long long seen;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(count) : "memory");
      (void)seen;
    }
    __threadfence();
    s_okw = ok;
  }
  __syncthreads();
  return s_okw != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long *count, unsigned long long target, int *err,
                                             unsigned long long limit_ns, bool acquire = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned long long *vc = count;
    volatile int *verr = err;
    __threadfence();
    atomicAdd(count, 1ull);
    int ok = 1;
    if (*vc < target) {
      const unsigned long long t0 = global_timer_ns();
      unsigned spins = 0;
      while (*vc < target) {
        if ((++spins & 63u) == 0u && (*verr || global_timer_ns() - t0 > limit_ns)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(8);
      }
    }
    if (ok && acquire) {
      // acquire: later loads of this CTA (ordered after it by the CTA barrier
      // below) see every write the other CTAs made before their arrival
      unsigned long long seen;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(count) : "memory");
      (void)seen;
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Step control of Algorithm 2 (the scalars one attempt reads and updates).
struct StepCtl {
  double eta, omega, inv_omega, tau, sigma, sum_eta;
  double dx2, dy2, inter, eta_bar;
  long long k, t, attempts;
  int cur, chunk_acc, status, const_step;
};

// Algorithm 2's test on the reductions of one attempt: eta_bar from the
// omega-weighted movement and the magnitude of the interaction term (a zero
// denominator gives eta_bar = +inf), acceptance iff eta <= eta_bar, then the
// next step size min(fr * eta_bar, fg * eta) with the factors
// fr = 1 - (k+1)^-0.3 and fg = 1 + (k+1)^-0.6 of the step count k before the
// attempt (k counted from 1).
__device__ __forceinline__ void step_update(StepCtl &c, double dx2, double dy2, double inter, double fr, double fg) {
  c.dx2 = dx2;
  c.dy2 = dy2;
  c.inter = inter;
  const double num = c.omega * dx2 + dy2 * c.inv_omega;
  const double den = 2.0 * fabs(inter);
  const double eta_bar = den > 0.0 ? num / den : INFINITY;
  const double e1 = fr * eta_bar;
  const double e2 = fg * c.eta;
  c.eta_bar = eta_bar;
  c.attempts += 1;
  if (!isfinite(num) || isnan(eta_bar) || isnan(inter)) {
    c.status = kNumErr;
    return;
  }
  if (c.const_step) {  // Section 2's baseline: a fixed eta, every step taken
    c.cur ^= 1;
    c.sum_eta += c.eta;
    c.k += 1;
    c.t += 1;
    c.chunk_acc += 1;
    return;
  }
  if (c.eta <= eta_bar) {
    c.cur ^= 1;
    c.sum_eta += c.eta;
    c.k += 1;
    c.t += 1;
    c.chunk_acc += 1;
  }
  c.eta = e1 < e2 ? e1 : e2;
  c.tau = c.eta * c.inv_omega;
  c.sigma = c.eta * c.omega;
}

__device__ __forceinline__ void load_step(const Scalars *s, StepCtl &c) {
  c.eta = s->eta;
  c.omega = s->omega;
  c.inv_omega = s->inv_omega;
  c.tau = s->tau;
  c.sigma = s->sigma;
  c.sum_eta = s->sum_eta;
  c.dx2 = s->dx2;
  c.dy2 = s->dy2;
  c.inter = s->inter;
  c.eta_bar = s->eta_bar;
  c.k = s->k;
  c.t = s->t;
  c.attempts = s->attempts;
  c.cur = s->cur;
  c.chunk_acc = s->chunk_acc;
  c.status = s->status;
  c.const_step = s->const_step;
}

__device__ __forceinline__ void store_step(Scalars *s, const StepCtl &c) {
  s->eta = c.eta;
  s->tau = c.tau;
  s->sigma = c.sigma;
  s->sum_eta = c.sum_eta;
  s->dx2 = c.dx2;
  s->dy2 = c.dy2;
  s->inter = c.inter;
  s->eta_bar = c.eta_bar;
  s->k = c.k;
  s->t = c.t;
  s->attempts = c.attempts;
  s->cur = c.cur;
  s->chunk_acc = c.chunk_acc;
  s->status = c.status;
}

// Shared-memory layout of the persistent step kernel: each warp has a slice
// of warp_bytes (its staging buffers, then the descriptors of its chunks of
// K^T and of K at byte offsets o_desc_p, o_desc_d).  grid == 0: not used.
struct PersistGeo {
  int32_t grid;   // CTAs (all co-resident)
  int32_t smem;   // dynamic shared memory per CTA
  int32_t warp_bytes;
  int32_t o_desc_p, o_desc_d;
  int32_t l1_gather;  // 1: gathers through L1 after acquiring barriers; 0: through L2 only
};

// Algorithm 2's factors 1 - (k+1)^-0.3 and 1 + (k+1)^-0.6 for the next
// eval_every steps k = fac_k0 + i + 1 (k counted from 1), by one CTA.
__device__ __forceinline__ void fill_step_factors(Scalars *s) {
  const long long k0 = s->fac_k0;
  const int ne = s->eval_every < kMaxEval ? s->eval_every : kMaxEval;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const double kk = (double)(k0 + i + 1);
    s->fac_tab[0][i] = 1.0 - pow(kk + 1.0, -0.3);
    s->fac_tab[1][i] = 1.0 + pow(kk + 1.0, -0.6);
  }
}

}  // namespace pdlp
