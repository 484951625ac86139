// Host-side planning shared by the library and its CPU tests: the warp-chunk
// schedule of a CSR matrix, the balanced assignment of chunks to the warps
// of the persistent kernel, the long rows of the preconditioning, and the
// tolerance, scale, stop and budget rules of the float32 iterative
// refinement.  Plain C++ (no CUDA headers), so that the
// tests can build it with the host compiler alone.
#pragma once

#include <stdint.h>

#include <vector>

namespace pdlp {

constexpr int kChunkNnz = 256;      // nonzeros staged per warp chunk
constexpr int kChunkRows = 32;      // rows per warp chunk (one epilogue lane per row)
constexpr int kSegNnz = kChunkNnz;  // rows longer than this are split across warps, one chunk each

// One warp's share of a CSR matrix.  Two kinds (with kSegNnz == kChunkNnz):
//   rows [row_begin, row_end) with at most kChunkNnz nonzeros and kChunkRows rows;
//   row_end < 0: a segment [nnz_begin, nnz_end) of long row -(row_end + 1).
// (A single row longer than kChunkNnz but not than kSegNnz would be a third
// kind, looped over by one warp; spmv_chunk still handles it.)
struct Chunk {
  int32_t row_begin, row_end, nnz_begin, nnz_end;
};

// A row longer than kSegNnz, processed by `nseg` warps (consecutive chunks).
struct LongRow {
  int32_t row, nseg, part_off, pad;
};

// Long rows of the Section 3.5 preconditioning, handled apart: the Ruiz
// maxima of rows longer than kMaxSeg nonzeros by one CTA per kMaxSeg-nonzero
// segment, combined with an atomic maximum on the bits (the numeric order
// for nonnegative doubles, so the result is the same in any order); the
// Pock-Chambolle l1 sums of rows longer than kLongScan on the host in CSR
// order, the order of the plain loop (one GPU thread, at GB300's float64 add
// rate, takes tens of milliseconds for a million terms).
constexpr int32_t kMaxSeg = 256;
constexpr int32_t kLongScan = 8192;
struct ScanSeg {
  int32_t row, k0, k1, pad;  // [k0, k1): a segment of row `row`
};
struct PrecondPlan {
  std::vector<ScanSeg> segK, segKT;    // kMaxSeg-nonzero segments of the rows of K, K^T longer than kMaxSeg
  std::vector<int32_t> longK, longKT;  // the rows of K, K^T longer than kLongScan
};
// From the host row starts of K (m rows) and K^T (n rows).
void plan_precondition(int32_t m, const int32_t *hrp, int32_t n, const int32_t *htrp, PrecondPlan &pp);

// Warp-chunk schedule of a CSR matrix with `rows` rows and host row_ptr rp:
// consecutive rows are grouped greedily into chunks of at most kChunkNnz
// nonzeros and kChunkRows rows; a row with more than kSegNnz nonzeros gets
// ceil(len / kSegNnz) segment chunks and a LongRow record (part_off = its
// first slot among nseg_total segment partials).
void build_schedule(int32_t rows, const int32_t *rp, std::vector<Chunk> &chunks,
                    std::vector<LongRow> &longrows, int32_t &nseg_total);

// Cost of one chunk in warp steps, the model behind the assignment: gathered
// entries per lane, twice the row-sum steps of the device's chunk_row_sums
// (float64 multiply-add plus shared-memory loads; at most kSegStepsHost, the
// segmented sum's), a fixed epilogue, and the combine of a long-row segment.
constexpr unsigned kSegStepsHost = 16;
double chunk_cost(const Chunk &c, const int32_t *rp);

// Balanced static assignment of chunks to nw warps (grids of nw /
// warps_per_cta CTAs): longest processing time first under chunk_cost, the
// least-loaded warp taking the next chunk, equal loads broken by rank, where
// rank r is warp (r % grid) * warps_per_cta + r / grid so that ties spread
// over the CTAs.  Warp w runs chunks idx[off[w] .. off[w+1]) in chunk order;
// cmax = the longest list.
void assign_chunks(const std::vector<Chunk> &chunks, const int32_t *rp, int nw, int warps_per_cta,
                   std::vector<int32_t> &idx, std::vector<int32_t> &off, int &cmax);

// Fixed-size slabs of a CSR matrix (the slab step kernels).  Slab s covers
// the nonzeros [kSlabNnz s, kSlabNnz (s + 1)) whatever the row boundaries,
// so every slab carries the same work however long the rows are; the value
// and index arrays are padded with zeros to nslab * kSlabNnz entries.  A row
// belongs to the slab that holds its first nonzero (an empty row to the slab
// holding position rp[r]); rows [first_row[s], first_row[s + 1]) belong to
// slab s.  A row that crosses one slab boundary and ends in the next slab
// is extended: the slab holding its start also reads its remaining nonzeros,
// and the next slab skips them (tail_split[s] = kSlabExtend - row,
// head_split[s+1] = kSlabSkip).  A row that reaches further is a split row:
// every slab it touches contributes one partial sum (slot part_off + s -
// s_first), and the last of them to finish adds the partials in slab order.
// head_split[s] is the split row that slab s's first nonzero continues (-1:
// the slab starts with a row start or holds no nonzero; kSlabSkip: an
// extended row's remainder), tail_split[s] the split row that starts in slab
// s and continues past its end (-1: none; <= kSlabExtend: the extended row
// kSlabExtend - tail_split[s]).  nslab = nnz / kSlabNnz + 1.
constexpr int kSlabNnz = 256;
constexpr int32_t kSlabSkip = -2;
constexpr int32_t kSlabExtend = -3;

struct SplitRow {
  int32_t row, s_first, s_last, part_off;
};

void build_slabs(int32_t rows, const int32_t *rp, std::vector<int32_t> &first_row, std::vector<int32_t> &head_split,
                 std::vector<int32_t> &tail_split, std::vector<SplitRow> &splits, int32_t &nparts);

// Scales of the correction problem from the primal / dual violations:
// dP = 1 / pv and dD = 1 / dv, each clipped to [1, dmax].
void refine_scales(double pv, double dv, double dmax, double *dP, double *dD);

// Tolerance of the next inner solve.  The error after a round is about the
// current error times the round's tolerance, so when 0.1 tol / current error
// (rel) is at least kInnerFloor (1e-6, what float32 reaches) the round uses
// it (capped at 0.1): the loosest solve expected to finish with a 10x
// margin; otherwise inner_tol.
constexpr double kInnerFloor = 1e-6;
double refine_round_tol(double rel, double tol, double inner_tol);

// A float32 round that divides the relative Eq. (15) error by less than this
// factor ends the float32 rounds: their corrections have stopped paying (the
// inner solves stall at what float32 resolves of the correction problem),
// and the solve finishes with float64 PDLP from the refined point.
constexpr double kRefineMinGain = 10.0;
// After the evaluation of round `round` (error `rel`; the previous round's
// `prev`, the start point's for round 1): 1 if the float32 rounds end here
// for the float64 finish (a round that gained less than kRefineMinGain, or
// the round cap), else 0.
int refine_finish_now(int round, double prev, double rel, int max_rounds);
// Limits of the next solve of one refinement (iterations, KKT passes, time in
// ns with 0 for none) from the caller's limits less what the earlier solves
// spent; returns 0 when all three have some left, else 1 (iterations), 2 (KKT
// passes) or 3 (time) for the first one spent.
int refine_remaining(long long iter_limit, long long kkt_limit, double time_limit_s, long long iters,
                     long long passes, double secs, long long out[3]);

}  // namespace pdlp
