// Host-side planning shared by the library and its CPU tests: the warp-chunk
// schedule of a CSR matrix, the balanced assignment of chunks to the warps
// of the persistent kernel, and the tolerance and scale rules of the
// float32 iterative refinement.  Plain C++ (no CUDA headers), so that the
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

}  // namespace pdlp
