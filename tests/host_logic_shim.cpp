// C entry points over the library's host-side planning (schedule.h) for the
// CPU tests; built by tests/test_host_logic.py with the host compiler.
#include <string.h>

#include <vector>

#include "schedule.h"

using namespace pdlp;

extern "C" int hl_build_schedule(int rows, const int32_t *rp, int32_t *chunks4, int cap_chunks, int32_t *long4,
                                 int cap_long, int32_t *counts /* nchunks, nlong, nseg_total */) {
  std::vector<Chunk> ch;
  std::vector<LongRow> lr;
  int32_t nseg = 0;
  build_schedule(rows, rp, ch, lr, nseg);
  counts[0] = (int32_t)ch.size();
  counts[1] = (int32_t)lr.size();
  counts[2] = nseg;
  if ((int)ch.size() > cap_chunks || (int)lr.size() > cap_long) return -1;
  memcpy(chunks4, ch.data(), sizeof(Chunk) * ch.size());
  memcpy(long4, lr.data(), sizeof(LongRow) * lr.size());
  return 0;
}

extern "C" double hl_chunk_cost(const int32_t *chunk4, const int32_t *rp) {
  Chunk c;
  memcpy(&c, chunk4, sizeof(c));
  return chunk_cost(c, rp);
}

extern "C" int hl_assign(int n, const int32_t *chunks4, const int32_t *rp, int nw, int wpc, int32_t *idx,
                         int32_t *off, int32_t *cmax) {
  std::vector<Chunk> ch((size_t)n);
  memcpy(ch.data(), chunks4, sizeof(Chunk) * (size_t)n);
  std::vector<int32_t> i, o;
  int cm = 0;
  assign_chunks(ch, rp, nw, wpc, i, o, cm);
  memcpy(idx, i.data(), sizeof(int32_t) * i.size());
  memcpy(off, o.data(), sizeof(int32_t) * o.size());
  *cmax = cm;
  return 0;
}

extern "C" double hl_round_tol(double rel, double tol, double inner) { return refine_round_tol(rel, tol, inner); }

extern "C" void hl_scales(double pv, double dv, double dmax, double *out) { refine_scales(pv, dv, dmax, out, out + 1); }

extern "C" int hl_finish_now(int round, double prev, double rel, int max_rounds) {
  return refine_finish_now(round, prev, rel, max_rounds);
}

extern "C" int hl_remaining(long long il, long long kl, double ts, long long it, long long kp, double secs,
                            long long *out) {
  return refine_remaining(il, kl, ts, it, kp, secs, out);
}

extern "C" int hl_build_slabs(int rows, const int32_t *rp, int32_t *first, int32_t *head, int32_t *tail,
                              int32_t *split4, int cap_split, int32_t *counts /* nslab, nsplit, nparts */) {
  std::vector<int32_t> f, h, t;
  std::vector<SplitRow> sp;
  int32_t nparts = 0;
  build_slabs(rows, rp, f, h, t, sp, nparts);
  counts[0] = (int32_t)h.size();
  counts[1] = (int32_t)sp.size();
  counts[2] = nparts;
  if ((int)sp.size() > cap_split) return -1;
  memcpy(first, f.data(), sizeof(int32_t) * f.size());
  memcpy(head, h.data(), sizeof(int32_t) * h.size());
  memcpy(tail, t.data(), sizeof(int32_t) * t.size());
  memcpy(split4, sp.data(), sizeof(SplitRow) * sp.size());
  return 0;
}

// plan_precondition on one matrix (m = rows, n = 0): segments as (row, k0, k1)
// triples and the rows whose l1 sums the host takes
extern "C" int hl_plan_precondition(int rows, const int32_t *rp, int32_t *seg3, int cap_seg, int32_t *longr,
                                    int cap_long, int32_t *counts /* nseg, nlong */) {
  PrecondPlan pp;
  const int32_t zero = 0;
  plan_precondition(rows, rp, 0, &zero, pp);
  counts[0] = (int32_t)pp.segK.size();
  counts[1] = (int32_t)pp.longK.size();
  if ((int)pp.segK.size() > cap_seg || (int)pp.longK.size() > cap_long) return -1;
  for (size_t i = 0; i < pp.segK.size(); ++i) {
    seg3[3 * i] = pp.segK[i].row;
    seg3[3 * i + 1] = pp.segK[i].k0;
    seg3[3 * i + 2] = pp.segK[i].k1;
  }
  for (size_t i = 0; i < pp.longK.size(); ++i) longr[i] = pp.longK[i];
  return 0;
}
