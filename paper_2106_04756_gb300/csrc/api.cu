// C ABI of the library (declared in include/pdlp.h): context set-up, the
// solve graph, float32 iterative refinement, inspection calls.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "presolve.cuh"
#include "refine.cuh"
#include "slab.cuh"
#include "solver.cuh"
#include "unroll.cuh"

using namespace pdlp;

namespace {

thread_local std::string g_last_error;

// Device buffers of one precision's iteration.
template <typename T>
struct Precision {
  bool ready = false;
  DevBuf val, tval;  // K~ and K~^T values (only for float: double uses the master copies)
  DevBuf cs, qs, ls, us, ylos;
  DevBuf vecs;       // every iterate vector, one allocation
  DevBuf parts, gkeys, ghist, xo, yo, tickets, normpart, trace;
  Mat<T> K, KT;
  Mat<T> KTb;       // KT with the second long-row buffers (the persistent evaluation's phase B)
  Problem<T> P;
  State<T> S;
  ScalarInit init{};
  double *normpart_ptr = nullptr;
  PersistGeo pg{};  // persistent step kernel layout (grid 0: one launch per half-step)
  PersistGeo pe{};  // persistent evaluation kernel layout (grid 0: the separate evaluation kernels)
  cudaGraphExec_t graph = nullptr;
  ~Precision() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

}  // namespace

namespace pdlp {
// Records a message returned by pdlp_last_error(NULL) on this thread.
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace pdlp

struct pdlp_ctx {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  pdlp_options opts;
  cudaStream_t st = nullptr;           // caller's stream
  cudaStream_t cap[4] = {nullptr, nullptr, nullptr, nullptr};  // capture streams (library-owned)
  std::string err;
  // matrix (float64 master copy, preconditioned in place)
  DevBuf rp, ci, val, trp, tci, tval, perm, rowid;  // rowid: row of every nonzero of K
  DevBuf blocksK, blocksKT, longK, longKT, segK, segKT, segcntK, segcntKT, lraccK, lraccKT;
  int32_t nlongK = 0, nlongKT = 0;
  int32_t nsegKT = 0;  // segment partials of K^T's long rows (per gathered vector)
  DevBuf wchunkK, woffK, wchunkKT, woffKT;  // chunk lists of the persistent kernel's warps
  int32_t cmaxK = 0, cmaxKT = 0, assign_nw = 0;
  // fixed-size slabs of K and K^T (the slab step kernels)
  DevBuf slabK, slabKT, splitK, splitKT, spartK, spartKT, scntK, scntKT, saccK, saccKT;
  int32_t nslabK = 0, nslabKT = 0, nsplitK = 0, nsplitKT = 0, ndeferK = 0, ndeferKT = 0;
  int32_t nblocksK = 0, nblocksKT = 0;
  std::vector<Chunk> hblocksK, hblocksKT;  // warp-chunk schedules
  // problem data
  DevBuf c, q, l, u, ylo;            // original space
  DevBuf cs, qs, ls, us, ylos;       // preconditioned (float64)
  DevBuf D1, D2, D1inv, D2inv;
  DevBuf xin, yin;                   // start point staging (original space)
  DevBuf mask;                       // inequality mask as given
  DevBuf scal;                       // Scalars
  double eta0 = 1.0;
  Precision<double> p64;
  Precision<float> p32;              // plain float32 solve of the LP itself
  Precision<float> pc32;             // float32 solves of refinement corrections
  RefineBuffers ref;
  UnrollBuffers unr;
  std::unique_ptr<Presolve> pre;     // presolve = 1: the original LP and the maps
  pdlp_ctx *inner = nullptr;         // presolve = 1: context of the reduced LP (null if none is left)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ~pdlp_ctx() {
    if (st) cudaStreamSynchronize(st);
    delete inner;
    for (auto &s : cap)
      if (s) cudaStreamDestroy(s);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

namespace {

int fail(pdlp_ctx *ctx, int code, const std::string &msg) {
  g_last_error = msg;
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(pdlp_ctx *ctx, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) return fail(ctx, PDLP_ERR_OOM, std::string(where) + ": out of device memory");
  return fail(ctx, PDLP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                                 \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

template <typename T>
T *dalloc(DevBuf &b, size_t count) {
  return reinterpret_cast<T *>(b.get(sizeof(T) * (count ? count : 1)));
}

__global__ void k_recip(const double *v, int64_t n, double *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0 / v[i];
}

__global__ void k_absmax_bits(const double *v, int64_t n, unsigned long long *out) {
  unsigned long long mx = 0ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v[i]));
    mx = b > mx ? b : mx;
  }
  atomicMax(out, mx);  // non-negative doubles order like their bit patterns
}

template <typename T>
int setup_matrix(pdlp_ctx *ctx, Mat<T> &K, Mat<T> &KT, const T *val, const T *tval) {
  K.rows = ctx->m;
  K.cols = ctx->n;
  K.rp = reinterpret_cast<const int32_t *>(ctx->rp.ptr());
  K.ci = reinterpret_cast<const int32_t *>(ctx->ci.ptr());
  K.val = val;
  K.chunks = reinterpret_cast<const Chunk *>(ctx->blocksK.ptr());
  K.nchunks = (int32_t)ctx->hblocksK.size();
  K.nblocks = ctx->nblocksK;
  K.longrows = reinterpret_cast<const LongRow *>(ctx->longK.ptr());
  K.seg_part = reinterpret_cast<double *>(ctx->segK.ptr());
  K.seg_cnt = reinterpret_cast<unsigned *>(ctx->segcntK.ptr());
  K.lr_acc = reinterpret_cast<double *>(ctx->lraccK.ptr());
  K.nlong = ctx->nlongK;
  K.wchunk = reinterpret_cast<const int32_t *>(ctx->wchunkK.ptr());
  K.woff = reinterpret_cast<const int32_t *>(ctx->woffK.ptr());
  K.assign_nw = ctx->assign_nw;
  {
    const int32_t *meta = reinterpret_cast<const int32_t *>(ctx->slabK.ptr());
    K.nslab = ctx->nslabK;
    K.nsplit = ctx->nsplitK;
    K.ndefer = ctx->ndeferK;
    K.slab_first = meta;
    K.slab_head = meta + K.nslab + 1;
    K.slab_tail = meta + 2 * K.nslab + 1;
    K.splits = reinterpret_cast<const SplitRow *>(ctx->splitK.ptr());
    K.split_part = reinterpret_cast<double *>(ctx->spartK.ptr());
    K.split_cnt = reinterpret_cast<unsigned *>(ctx->scntK.ptr());
    K.split_acc = reinterpret_cast<double *>(ctx->saccK.ptr());
  }
  KT.rows = ctx->n;
  KT.cols = ctx->m;
  KT.rp = reinterpret_cast<const int32_t *>(ctx->trp.ptr());
  KT.ci = reinterpret_cast<const int32_t *>(ctx->tci.ptr());
  KT.val = tval;
  KT.chunks = reinterpret_cast<const Chunk *>(ctx->blocksKT.ptr());
  KT.nchunks = (int32_t)ctx->hblocksKT.size();
  KT.nblocks = ctx->nblocksKT;
  KT.longrows = reinterpret_cast<const LongRow *>(ctx->longKT.ptr());
  KT.seg_part = reinterpret_cast<double *>(ctx->segKT.ptr());
  KT.seg_cnt = reinterpret_cast<unsigned *>(ctx->segcntKT.ptr());
  KT.lr_acc = reinterpret_cast<double *>(ctx->lraccKT.ptr());
  KT.nlong = ctx->nlongKT;
  KT.wchunk = reinterpret_cast<const int32_t *>(ctx->wchunkKT.ptr());
  KT.woff = reinterpret_cast<const int32_t *>(ctx->woffKT.ptr());
  KT.assign_nw = ctx->assign_nw;
  {
    const int32_t *meta = reinterpret_cast<const int32_t *>(ctx->slabKT.ptr());
    KT.nslab = ctx->nslabKT;
    KT.nsplit = ctx->nsplitKT;
    KT.ndefer = ctx->ndeferKT;
    KT.slab_first = meta;
    KT.slab_head = meta + KT.nslab + 1;
    KT.slab_tail = meta + 2 * KT.nslab + 1;
    KT.splits = reinterpret_cast<const SplitRow *>(ctx->splitKT.ptr());
    KT.split_part = reinterpret_cast<double *>(ctx->spartKT.ptr());
    KT.split_cnt = reinterpret_cast<unsigned *>(ctx->scntKT.ptr());
    KT.split_acc = reinterpret_cast<double *>(ctx->saccKT.ptr());
  }
  return PDLP_OK;
}

// The step engine of a context (option `persistent`): 2 = slab kernels;
// 0 = warp-chunk kernels, one launch per half-step; 1 (default) and 3 = the
// persistent warp-chunk kernel where its layout fits, else 0.  Measured per
// step attempt on GB300 (float64 / float32): the persistent kernel 170 /
// 112 us on the 1M-node PageRank LP and 42.5 / 29.1 us on the 100k x 250k LP,
// the slab kernels 217 / 139 and 66 / 46 us, so the default never picks them.
constexpr double kL1GatherBytes = 96e6;  // working set above which the persistent kernel gathers through L1
int use_slab_engine(const pdlp_ctx *ctx, int elem_bytes) {
  (void)elem_bytes;
  return ctx->opts.persistent == 2;
}

// Allocates the iterate state of one precision and captures its solve graph
// on the problem `P` (already filled in).
template <typename T>
int setup_state(pdlp_ctx *ctx, Precision<T> &pr, double tol, const double *tol_dev = nullptr,
                int stall_evals = 0, const long long *lim_dev = nullptr) {
  const int n = ctx->n, m = ctx->m, N = n + m;
  const size_t nv = 2 * (size_t)n + 2 * (size_t)m + 2 * (size_t)m + 2 * (size_t)n + 2 * (size_t)m +
                    (size_t)n + (size_t)m + 2 * (size_t)n + (size_t)m;
  T *v = dalloc<T>(pr.vecs, nv);
  if (!v) return fail(ctx, PDLP_ERR_OOM, "state allocation failed");
  CK(cudaMemsetAsync(v, 0, sizeof(T) * nv, ctx->st), "memset state");
  State<T> &S = pr.S;
  T *p = v;
  auto take = [&](size_t k) { T *r = p; p += k; return r; };
  S.x[0] = take(n); S.x[1] = take(n);
  S.y[0] = take(m); S.y[1] = take(m);
  S.Kx[0] = take(m); S.Kx[1] = take(m);
  S.xs[0] = take(n); S.xs[1] = take(n);
  S.ys[0] = take(m); S.ys[1] = take(m);
  S.x0 = take(n); S.y0 = take(m);
  S.KTy_cur = take(n); S.KTys = take(n);
  S.Kxbar = take(m);
  S.eta_log = nullptr;
  // step engine: the slab kernels, the persistent warp-chunk kernel or the
  // per-launch warp-chunk kernels (the Malitsky-Pock line search runs on the
  // last)
  const int slab = ctx->opts.step_policy != 2 && use_slab_engine(ctx, (int)sizeof(T));
  pr.K.slab_on = pr.KT.slab_on = slab;
  if (slab) CK(plan_slab_grid<T>(pr.K, pr.KT), "slab grid");
  const int persist_mode = (ctx->opts.step_policy == 2 || slab || ctx->opts.persistent == 0) ? 0 : 1;
  // gathers through L1 when one attempt's working set exceeds L2 (see persistent.cu)
  const double ws = 2.0 * (double)ctx->nnz * (4.0 + sizeof(T)) + 4.0 * ((double)ctx->m + ctx->n) +
                    (double)sizeof(T) * (9.0 * ctx->n + 10.0 * ctx->m);
  const int l1g = ctx->opts.persistent == 4 ? 1 : (ctx->opts.persistent == 3 ? 0 : (ws > kL1GatherBytes ? 1 : 0));
  CK(persist_plan<T>(ctx->cmaxKT, ctx->cmaxK, ctx->assign_nw, persist_mode, l1g, &pr.pg), "persistent kernel layout");
  CK(eval_plan<T>(pr.pg, ctx->cmaxKT, ctx->cmaxK, &pr.pe), "persistent evaluation layout");
  // K^T for the persistent evaluation's second walk: segment partials in the
  // second half of the (two-vector) area, the second set of counters, and
  // epilogue slots 4..7 of each long row
  pr.KTb = pr.KT;
  pr.KTb.seg_part = pr.KT.seg_part + ctx->nsegKT;
  pr.KTb.seg_cnt = pr.KT.seg_cnt + ctx->nlongKT;
  pr.KTb.lr_acc = pr.KT.lr_acc + 4;
  const size_t nsp = (size_t)slab_ctas(ctx->nslabKT), nsd = 2 * (size_t)slab_ctas(ctx->nslabK);
  const size_t np = (size_t)ctx->nblocksKT + 2 * (size_t)ctx->nblocksK + 8 * (size_t)ctx->nblocksKT +
                    8 * (size_t)ctx->nblocksK + 3 * (size_t)pr.pg.grid + nsp + nsd + 16 * (size_t)pr.pe.grid + 16;
  double *parts = dalloc<double>(pr.parts, np);
  if (!parts) return fail(ctx, PDLP_ERR_OOM, "partials allocation failed");
  S.part_p = parts;
  S.part_d = S.part_p + ctx->nblocksKT;
  S.part_ec = S.part_d + 2 * (size_t)ctx->nblocksK;
  S.part_er = S.part_ec + 8 * (size_t)ctx->nblocksKT;
  S.part_cp = S.part_er + 8 * (size_t)ctx->nblocksK;
  S.part_sp = S.part_cp + 3 * (size_t)pr.pg.grid;
  S.part_sd = S.part_sp + nsp;
  S.part_ce = S.part_sd + nsd;
  // fixed tickets, then one counter per group of 32 evaluation CTAs
  const size_t nticket = kNumTickets + ((size_t)ctx->nblocksKT + 31) / 32 + ((size_t)ctx->nblocksK + 31) / 32;
  S.tickets = dalloc<unsigned>(pr.tickets, nticket);
  S.gtickets = S.tickets ? S.tickets + kNumTickets : nullptr;
  S.gkeys = dalloc<unsigned>(pr.gkeys, (size_t)kGapSlots * N);
  // the gap histograms, then their bitmaps of nonempty buckets (1 bit each)
  const size_t ghist_n = (size_t)kGapSlots * kGapBuckets * 3 + (size_t)kGapSlots * kGapBuckets / 64;
  S.ghist = dalloc<double>(pr.ghist, ghist_n);
  S.gmask = S.ghist ? reinterpret_cast<unsigned *>(S.ghist + (size_t)kGapSlots * kGapBuckets * 3) : nullptr;
  S.xo = dalloc<double>(pr.xo, n);
  S.yo = dalloc<double>(pr.yo, m);
  S.s = reinterpret_cast<Scalars *>(ctx->scal.ptr());
  S.trace = dalloc<double>(pr.trace, (size_t)kTraceCap * kTraceLen);
  if (!S.trace) return fail(ctx, PDLP_ERR_OOM, "trace allocation failed");
  double *normpart = dalloc<double>(pr.normpart, 4 * 152 + 8);
  if (!S.tickets || !S.gkeys || !S.ghist || !S.xo || !S.yo || !normpart)
    return fail(ctx, PDLP_ERR_OOM, "state allocation failed");
  CK(cudaMemsetAsync(S.tickets, 0, sizeof(unsigned) * nticket, ctx->st), "memset");
  CK(cudaMemsetAsync(S.ghist, 0, sizeof(double) * ghist_n, ctx->st), "memset");
  CK(cudaMemsetAsync(normpart, 0, sizeof(double) * (4 * 152 + 8), ctx->st), "memset");
  CK(set_kernel_attributes<T>(), "kernel attributes");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  const pdlp_options &o = ctx->opts;
  ScalarInit in{};
  in.eta0 = ctx->eta0;
  in.rel_tol = tol;
  in.tol_dev = tol_dev;
  in.stall_evals = stall_evals;
  in.lim_dev = lim_dev;
  in.beta_suff = o.beta_suff;
  in.beta_nec = o.beta_nec;
  in.beta_art = o.beta_art;
  in.pw_theta = o.pw_smoothing;
  in.eps_zero = o.eps_zero;
  in.iter_limit = o.iter_limit;
  in.attempt_limit = o.kkt_pass_limit;
  in.time_limit_ns = o.time_limit_s > 0 ? (unsigned long long)(o.time_limit_s * 1e9) : 0ull;
  in.wait_ns = o.wait_limit_us == 0 ? kBarrierTimeoutNs
                                    : 1000ull * (unsigned long long)(o.wait_limit_us > 0 ? (long long)o.wait_limit_us
                                                                                       : -(long long)o.wait_limit_us);
  in.wait_extra = o.wait_limit_us < 0 ? 1 : 0;
  in.eval_every = o.eval_every;
  in.adaptive_restart = o.adaptive_restart;
  in.pw_update = o.pw_update;
  in.const_step = o.step_policy == 1 ? 1 : 0;
  in.omega0 = o.omega0;
  in.restart_to_current = o.restart_to_current;
  in.mp = o.step_policy == 2 ? 1 : 0;
  in.mp_breaking = o.mp_breaking;
  in.mp_downscaling = o.mp_downscaling;
  in.mp_interpolation = o.mp_interpolation;
  if (in.const_step) {  // eta = 0.9 / ||K~||_2 (power iteration; the state vectors are scratch here)
    double kn = 0.0;
    CK(power_norm<T>(pr.K, pr.KT, 200, S.xs[0], S.Kx[1], S.xs[1], normpart, ctx->st, &kn), "power iteration");
    in.eta0 = kn > 0.0 ? 0.9 / kn : 1.0;
  }
  pr.init = in;
  pr.normpart_ptr = normpart;
  if (!o.use_graph) {
    pr.ready = true;
    return PDLP_OK;
  }
  CK(build_solve_graph<T>(pr.K, pr.KT, pr.KTb, pr.P, pr.S, in, o.primal_importance, normpart,
                          reinterpret_cast<const double *>(ctx->xin.ptr()),
                          reinterpret_cast<const double *>(ctx->yin.ptr()), 152, pr.pg, pr.pe, ctx->cap[0],
                          ctx->cap[1], ctx->cap[2], ctx->cap[3], &pr.graph),
     "graph capture");
  pr.ready = true;
  return PDLP_OK;
}

// Fills the float64 problem view with the context's own LP.
void fill_problem64(pdlp_ctx *ctx, Problem<double> &P) {
  P.m = ctx->m;
  P.n = ctx->n;
  P.cs = reinterpret_cast<const double *>(ctx->cs.ptr());
  P.qs = reinterpret_cast<const double *>(ctx->qs.ptr());
  P.ls = reinterpret_cast<const double *>(ctx->ls.ptr());
  P.us = reinterpret_cast<const double *>(ctx->us.ptr());
  P.ylos = reinterpret_cast<const double *>(ctx->ylos.ptr());
  P.c = reinterpret_cast<const double *>(ctx->c.ptr());
  P.q = reinterpret_cast<const double *>(ctx->q.ptr());
  P.l = reinterpret_cast<const double *>(ctx->l.ptr());
  P.u = reinterpret_cast<const double *>(ctx->u.ptr());
  P.ylo = reinterpret_cast<const double *>(ctx->ylo.ptr());
  P.D1 = reinterpret_cast<const double *>(ctx->D1.ptr());
  P.D2 = reinterpret_cast<const double *>(ctx->D2.ptr());
  P.D1inv = reinterpret_cast<const double *>(ctx->D1inv.ptr());
  P.D2inv = reinterpret_cast<const double *>(ctx->D2inv.ptr());
}

// PDLP_FP32_REFINE: the device limits shared by the inner float32 solves and
// the float64 finish (refine.cu), set to the caller's limits until a solve
// writes what is left of them.
const long long *refine_limits(pdlp_ctx *ctx) {
  if (ctx->opts.precision != PDLP_FP32_REFINE) return nullptr;
  long long *d = refine_limits_dev(ctx->ref);
  if (!d) return nullptr;
  const pdlp_options &o = ctx->opts;
  const long long full[4] = {o.iter_limit, o.kkt_pass_limit,
                             o.time_limit_s > 0 ? (long long)(o.time_limit_s * 1e9) : 0ll, 0ll};
  if (cudaMemcpy(d, full, sizeof(full), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  return d;
}

int setup_fp64(pdlp_ctx *ctx) {
  Precision<double> &pr = ctx->p64;
  if (pr.ready) return PDLP_OK;
  setup_matrix<double>(ctx, pr.K, pr.KT, reinterpret_cast<const double *>(ctx->val.ptr()),
                       reinterpret_cast<const double *>(ctx->tval.ptr()));
  fill_problem64(ctx, pr.P);
  const long long *lim = refine_limits(ctx);
  if (ctx->opts.precision == PDLP_FP32_REFINE && !lim) return fail(ctx, PDLP_ERR_OOM, "limits allocation failed");
  return setup_state<double>(ctx, pr, ctx->opts.rel_tol, nullptr, 0, lim);
}

// float32 copies of K~, K~^T (shared by the plain float32 and the refinement paths)
int ensure_float_matrix(pdlp_ctx *ctx, Precision<float> &pr, Precision<float> *share) {
  const float *v = nullptr, *tv = nullptr;
  if (share && share->val.ptr()) {
    v = reinterpret_cast<const float *>(share->val.ptr());
    tv = reinterpret_cast<const float *>(share->tval.ptr());
  } else {
    float *a = dalloc<float>(pr.val, ctx->nnz + kSlabNnz), *b = dalloc<float>(pr.tval, ctx->nnz + kSlabNnz);
    if (!a || !b) return fail(ctx, PDLP_ERR_OOM, "float matrix allocation failed");
    CK(cudaMemsetAsync(a + ctx->nnz, 0, sizeof(float) * kSlabNnz, ctx->st), "pad");
    CK(cudaMemsetAsync(b + ctx->nnz, 0, sizeof(float) * kSlabNnz, ctx->st), "pad");
    CK(to_float(reinterpret_cast<const double *>(ctx->val.ptr()), ctx->nnz, a, ctx->st), "to_float");
    CK(to_float(reinterpret_cast<const double *>(ctx->tval.ptr()), ctx->nnz, b, ctx->st), "to_float");
    v = a;
    tv = b;
  }
  setup_matrix<float>(ctx, pr.K, pr.KT, v, tv);
  return PDLP_OK;
}

int setup_fp32(pdlp_ctx *ctx) {
  Precision<float> &pr = ctx->p32;
  if (pr.ready) return PDLP_OK;
  int rc = ensure_float_matrix(ctx, pr, &ctx->pc32);
  if (rc) return rc;
  const int n = ctx->n, m = ctx->m;
  float *cs = dalloc<float>(pr.cs, n), *qs = dalloc<float>(pr.qs, m), *ls = dalloc<float>(pr.ls, n),
        *us = dalloc<float>(pr.us, n), *ylos = dalloc<float>(pr.ylos, m);
  if (!cs || !qs || !ls || !us || !ylos) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
  CK(to_float(reinterpret_cast<const double *>(ctx->cs.ptr()), n, cs, ctx->st), "to_float");
  CK(to_float(reinterpret_cast<const double *>(ctx->qs.ptr()), m, qs, ctx->st), "to_float");
  CK(to_float(reinterpret_cast<const double *>(ctx->ls.ptr()), n, ls, ctx->st), "to_float");
  CK(to_float(reinterpret_cast<const double *>(ctx->us.ptr()), n, us, ctx->st), "to_float");
  CK(to_float(reinterpret_cast<const double *>(ctx->ylos.ptr()), m, ylos, ctx->st), "to_float");
  Problem<double> P64;
  fill_problem64(ctx, P64);
  Problem<float> &P = pr.P;
  P.m = m;
  P.n = n;
  P.cs = cs; P.qs = qs; P.ls = ls; P.us = us; P.ylos = ylos;
  P.c = P64.c; P.q = P64.q; P.l = P64.l; P.u = P64.u; P.ylo = P64.ylo;
  P.D1 = P64.D1; P.D2 = P64.D2;
  P.D1inv = P64.D1inv; P.D2inv = P64.D2inv;
  return setup_state<float>(ctx, pr, ctx->opts.rel_tol);
}

int setup_refine(pdlp_ctx *ctx) {
  Precision<float> &pr = ctx->pc32;
  if (pr.ready) return PDLP_OK;
  int rc = ensure_float_matrix(ctx, pr, &ctx->p32);
  if (rc) return rc;
  rc = setup_fp64(ctx);  // float64 K~ products for the residuals
  if (rc) return rc;
  CK(refine_alloc(ctx->ref, ctx->m, ctx->n, ctx->nblocksK, ctx->nblocksKT), "refinement allocation");
  Problem<double> P64;
  fill_problem64(ctx, P64);
  pr.P = refine_problem(ctx->ref, P64);
  double *tol_dev = reinterpret_cast<double *>(ctx->ref.tol.ptr());
  CK(cudaMemcpy(tol_dev, &ctx->opts.inner_tol, sizeof(double), cudaMemcpyHostToDevice), "tolerance");
  // an inner solve that stops improving (the float32 floor of a
  // correction problem) returns to the outer loop after 250 evaluations
  // (10,000 iterations) without a 10% gain; windows of 50 cut off plateaus
  // that restarted PDHG passes through on its way (measured on PageRank)
  return setup_state<float>(ctx, pr, ctx->opts.inner_tol, tol_dev, 250, refine_limits(ctx));
}

void read_result(const Scalars &s, double seconds, pdlp_result *res) {
  memset(res, 0, sizeof(*res));
  res->status = s.status;
  res->returned_average = s.ret_which;
  res->iters = s.k;
  res->kkt_passes = s.attempts;
  res->restarts = s.restarts;
  const double *k = s.kkt[s.ret_which];
  res->primal_obj = k[0];
  res->dual_obj = k[1];
  res->gap = k[2];
  res->pres = k[3];
  res->dres = k[4];
  res->rel_gap = k[5];
  res->rel_pres = k[6];
  res->rel_dres = k[7];
  res->seconds = seconds;
  res->step_size = s.eta;
  res->primal_weight = s.omega;
}

// Step engine of one precision (pdlp_result.engine).
template <typename T>
int engine_of(const Precision<T> &pr) {
  return pr.K.slab_on ? 2 : (pr.pg.grid > 0 ? 1 : 0);
}

// Launches one precision's solve graph from the staged start point.
template <typename T>
int run_graph(pdlp_ctx *ctx, Precision<T> &pr, Scalars *hs) {
  if (!ctx->opts.use_graph) {
    CK(run_stepped<T>(pr.K, pr.KT, pr.P, pr.S, pr.init, ctx->opts.primal_importance, pr.normpart_ptr,
                      reinterpret_cast<const double *>(ctx->xin.ptr()),
                      reinterpret_cast<const double *>(ctx->yin.ptr()), 152, pr.pg, ctx->st, hs),
       "stepped solve");
  } else {
    CK(cudaGraphLaunch(pr.graph, ctx->st), "graph launch");
    CK(cudaMemcpyAsync(hs, pr.S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st), "scalars");
    CK(cudaStreamSynchronize(ctx->st), "solve");
  }
  if (hs->status == kWaitTimeout || hs->err)
    return fail(ctx, PDLP_ERR_TIMEOUT, "a grid-wide barrier of the persistent step kernel timed out");
  return PDLP_OK;
}

int stage_start(pdlp_ctx *ctx, const double *x0, const double *y0) {
  double *xi = reinterpret_cast<double *>(ctx->xin.ptr()), *yi = reinterpret_cast<double *>(ctx->yin.ptr());
  if (x0) CK(cudaMemcpyAsync(xi, x0, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st), "x0");
  else CK(cudaMemsetAsync(xi, 0, sizeof(double) * ctx->n, ctx->st), "x0");
  if (y0) CK(cudaMemcpyAsync(yi, y0, sizeof(double) * ctx->m, cudaMemcpyDefault, ctx->st), "y0");
  else CK(cudaMemsetAsync(yi, 0, sizeof(double) * ctx->m, ctx->st), "y0");
  return PDLP_OK;
}

int check_options(const pdlp_options *o, std::string &why) {
  if (!(o->rel_tol >= 0.0)) { why = "rel_tol must be >= 0"; return 0; }
  if (o->precision < PDLP_FP64 || o->precision > PDLP_FP32_REFINE) { why = "unknown precision"; return 0; }
  if (o->eval_every < 1 || o->eval_every > kMaxEval) { why = "eval_every must be in [1, 256]"; return 0; }
  if (o->persistent < 0 || o->persistent > 4) { why = "persistent must be 0, 1, 2, 3 or 4"; return 0; }
  if (o->step_policy < 0 || o->step_policy > 2) { why = "step_policy must be 0, 1 or 2"; return 0; }
  if (o->restart_to_current < 0 || o->restart_to_current > 1) { why = "restart_to_current must be 0 or 1"; return 0; }
  if (o->step_policy == 2 && o->unroll_T > 0) { why = "step_policy 2 does not combine with unroll_T > 0"; return 0; }
  if (!(o->mp_breaking >= 0.0) || !isfinite(o->mp_breaking)) { why = "mp_breaking must be finite and >= 0"; return 0; }
  if (!(o->mp_downscaling > 0.0 && o->mp_downscaling < 1.0)) { why = "mp_downscaling must be in (0, 1)"; return 0; }
  if (!(o->mp_interpolation >= 0.0 && o->mp_interpolation <= 1.0)) { why = "mp_interpolation must be in [0, 1]"; return 0; }
  if (!(o->omega0 >= 0.0) || !isfinite(o->omega0)) { why = "omega0 must be finite and >= 0"; return 0; }
  if (o->presolve < 0 || o->presolve > 1) { why = "presolve must be 0 or 1"; return 0; }
  if (o->presolve && o->unroll_T > 0) { why = "presolve does not combine with unroll_T > 0"; return 0; }
  if (o->ruiz_iters < 0) { why = "ruiz_iters must be >= 0"; return 0; }
  if (o->iter_limit < 0 || o->kkt_pass_limit < 0) { why = "limits must be >= 0"; return 0; }
  if (!(o->primal_importance > 0.0)) { why = "primal_importance must be > 0"; return 0; }
  if (!(o->pw_smoothing >= 0.0 && o->pw_smoothing <= 1.0)) { why = "pw_smoothing must be in [0, 1]"; return 0; }
  return 1;
}

// presolve = 1: the reductions of presolve.cu on the original LP, then an
// inner context (presolve = 0) for what is left.
int create_presolved(const pdlp_csr *K, const double *c, const double *q, const double *l, const double *u,
                     const uint8_t *ineq_mask, const pdlp_options &o, pdlp_ctx **out) {
  std::unique_ptr<pdlp_ctx> hold(new pdlp_ctx());
  pdlp_ctx *ctx = hold.get();
  const int m = K->m, n = K->n;
  const int64_t nnz = K->nnz;
  ctx->m = m;
  ctx->n = n;
  ctx->nnz = nnz;
  ctx->opts = o;
  ctx->st = reinterpret_cast<cudaStream_t>(o.stream);
  cudaStream_t st = ctx->st;
  CK(cudaEventCreate(&ctx->ev0), "event");
  CK(cudaEventCreate(&ctx->ev1), "event");
  ctx->pre.reset(new Presolve());
  Presolve &pre = *ctx->pre;
  pre.m0 = m;
  pre.n0 = n;
  pre.nnz0 = nnz;
  int32_t *rp = dalloc<int32_t>(pre.rp0, (size_t)m + 1), *ci = dalloc<int32_t>(pre.ci0, nnz);
  int32_t *rowid = dalloc<int32_t>(pre.rowid0, nnz);
  double *val = dalloc<double>(pre.val0, nnz), *dc = dalloc<double>(pre.c0, n), *dq = dalloc<double>(pre.q0, m),
         *dl = dalloc<double>(pre.l0, n), *du = dalloc<double>(pre.u0, n);
  uint8_t *mask = dalloc<uint8_t>(pre.ineq0, m);
  double *xin = dalloc<double>(ctx->xin, n), *yin = dalloc<double>(ctx->yin, m);
  DevBuf errbuf;
  unsigned *derr = dalloc<unsigned>(errbuf, 1), herr = 0;
  if (!rp || !ci || !rowid || !val || !dc || !dq || !dl || !du || !mask || !xin || !yin || !derr)
    return fail(ctx, PDLP_ERR_OOM, "input allocation failed");
  CK(cudaMemcpyAsync(rp, K->row_ptr, sizeof(int32_t) * ((size_t)m + 1), cudaMemcpyDefault, st), "copy row_ptr");
  if (nnz > 0) {
    CK(cudaMemcpyAsync(ci, K->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDefault, st), "copy col_idx");
    CK(cudaMemcpyAsync(val, K->val, sizeof(double) * nnz, cudaMemcpyDefault, st), "copy val");
  }
  CK(cudaMemcpyAsync(dc, c, sizeof(double) * n, cudaMemcpyDefault, st), "copy c");
  CK(cudaMemcpyAsync(dq, q, sizeof(double) * m, cudaMemcpyDefault, st), "copy q");
  CK(cudaMemcpyAsync(dl, l, sizeof(double) * n, cudaMemcpyDefault, st), "copy l");
  CK(cudaMemcpyAsync(du, u, sizeof(double) * n, cudaMemcpyDefault, st), "copy u");
  CK(cudaMemcpyAsync(mask, ineq_mask, sizeof(uint8_t) * m, cudaMemcpyDefault, st), "copy ineq_mask");
  CK(validate(m, n, nnz, rp, ci, val, dc, dq, dl, du, rowid, derr, &herr, st), "validate");
  if (herr) return fail(ctx, PDLP_ERR_INVALID_ARG, validate_message(herr));
  CK(presolve_run(pre, st), "presolve");
  pre.rowid0.reset();
  pre.ttmp.reset();
  if (pre.status == kPreReduced) {
    pdlp_csr K1{pre.m1, pre.n1, pre.nnz1, reinterpret_cast<const int32_t *>(pre.rp1.ptr()),
                reinterpret_cast<const int32_t *>(pre.ci1.ptr()), reinterpret_cast<const double *>(pre.val1.ptr())};
    pdlp_options oi = o;
    oi.presolve = 0;
    const int rc = pdlp_create(&K1, reinterpret_cast<const double *>(pre.c1.ptr()),
                               reinterpret_cast<const double *>(pre.q1.ptr()),
                               reinterpret_cast<const double *>(pre.l1.ptr()),
                               reinterpret_cast<const double *>(pre.u1.ptr()),
                               reinterpret_cast<const uint8_t *>(pre.ineq1.ptr()), &oi, &ctx->inner);
    if (rc) return fail(ctx, rc, std::string("reduced LP: ") + pdlp_last_error(nullptr));
    for (DevBuf *b : {&pre.rp1, &pre.ci1, &pre.val1, &pre.c1, &pre.q1, &pre.l1, &pre.u1, &pre.ineq1}) b->reset();
  }
  *out = hold.release();
  return PDLP_OK;
}

int solve_presolved(pdlp_ctx *ctx, const double *x0, const double *y0, double *x_out, double *y_out,
                    pdlp_result *res) {
  Presolve &pre = *ctx->pre;
  cudaStream_t st = ctx->st;
  const int m = ctx->m, n = ctx->n;
  double *xin = reinterpret_cast<double *>(ctx->xin.ptr()), *yin = reinterpret_cast<double *>(ctx->yin.ptr());
  double *x1 = reinterpret_cast<double *>(pre.x1.ptr()), *y1 = reinterpret_cast<double *>(pre.y1.ptr());
  pdlp_result r;
  memset(&r, 0, sizeof(r));
  CK(cudaEventRecord(ctx->ev0, st), "event");
  if (pre.status == kPreReduced) {
    const double *sx = nullptr, *sy = nullptr;
    if (x0 || y0) {
      if (x0) CK(cudaMemcpyAsync(xin, x0, sizeof(double) * n, cudaMemcpyDefault, st), "x0");
      if (y0) CK(cudaMemcpyAsync(yin, y0, sizeof(double) * m, cudaMemcpyDefault, st), "y0");
      CK(presolve_map_start(pre, x0 ? xin : nullptr, y0 ? yin : nullptr, st), "start");
      sx = x1;
      sy = y1;
    }
    const int rc = pdlp_solve(ctx->inner, sx, sy, x1, y1, &r);
    if (rc) return fail(ctx, rc, std::string("reduced LP: ") + pdlp_last_error(ctx->inner));
  } else {
    CK(cudaMemsetAsync(x1, 0, sizeof(double) * pre.n1, st), "x1");
    CK(cudaMemsetAsync(y1, 0, sizeof(double) * pre.m1, st), "y1");
    r.status = pre.status;
  }
  double kkt[8];
  CK(postsolve(pre, x1, y1, xin, yin, kkt, st), "postsolve");
  CK(cudaEventRecord(ctx->ev1, st), "event");
  r.primal_obj = kkt[0];
  r.dual_obj = kkt[1];
  r.gap = kkt[2];
  r.pres = kkt[3];
  r.dres = kkt[4];
  r.rel_gap = kkt[5];
  r.rel_pres = kkt[6];
  r.rel_dres = kkt[7];
  if (x_out) CK(cudaMemcpyAsync(x_out, xin, sizeof(double) * n, cudaMemcpyDefault, st), "x_out");
  if (y_out) CK(cudaMemcpyAsync(y_out, yin, sizeof(double) * m, cudaMemcpyDefault, st), "y_out");
  CK(cudaStreamSynchronize(st), "solve");
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "event");
  r.seconds = ms * 1e-3;
  if (res) *res = r;
  return PDLP_OK;
}

}  // namespace

// ===================================================================== ABI

extern "C" int pdlp_default_options(pdlp_options *o) {
  if (!o) return fail(nullptr, PDLP_ERR_INVALID_ARG, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->rel_tol = 1e-8;
  o->iter_limit = 1000000;
  o->kkt_pass_limit = 4000000;
  o->time_limit_s = 3600.0;
  o->precision = PDLP_FP64;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->eval_every = 40;
  o->adaptive_restart = 1;
  o->pw_update = 1;
  o->pw_smoothing = 0.5;
  o->primal_importance = 1.0;
  o->beta_suff = 0.9;
  o->beta_nec = 0.1;
  o->beta_art = 0.5;
  o->eps_zero = 1e-10;
  o->inner_tol = 1e-7;
  o->refine_rounds = 12;
  o->unroll_T = 0;
  o->ckpt_every = 50;
  o->use_graph = 1;
  o->persistent = 1;
  o->step_policy = 0;
  o->omega0 = 0.0;
  o->presolve = 0;
  o->restart_to_current = 1;
  o->mp_breaking = 1.0;
  o->mp_downscaling = 0.5;
  o->mp_interpolation = 0.4;
  o->stream = nullptr;
  return PDLP_OK;
}

extern "C" int pdlp_create(const pdlp_csr *K, const double *c, const double *q, const double *l,
                           const double *u, const uint8_t *ineq_mask, const pdlp_options *opts,
                           pdlp_ctx **out) {
  if (out) *out = nullptr;
  if (!K || !c || !q || !l || !u || !ineq_mask || !out)
    return fail(nullptr, PDLP_ERR_INVALID_ARG, "NULL argument");
  if (K->m < 1 || K->n < 1 || K->nnz < 0 || K->nnz > 2147483647ll || !K->row_ptr ||
      (K->nnz > 0 && (!K->col_idx || !K->val)))
    return fail(nullptr, PDLP_ERR_INVALID_ARG, "bad CSR dimensions (m, n >= 1, 0 <= nnz < 2^31)");
  pdlp_options o;
  if (opts) o = *opts; else pdlp_default_options(&o);
  std::string why;
  if (!check_options(&o, why)) return fail(nullptr, PDLP_ERR_INVALID_ARG, why);
  if (o.presolve) return create_presolved(K, c, q, l, u, ineq_mask, o, out);
  std::unique_ptr<pdlp_ctx> hold(new pdlp_ctx());
  pdlp_ctx *ctx = hold.get();
  ctx->m = K->m;
  ctx->n = K->n;
  ctx->nnz = K->nnz;
  ctx->opts = o;
  ctx->st = reinterpret_cast<cudaStream_t>(o.stream);
  for (auto &s : ctx->cap) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
  CK(cudaEventCreate(&ctx->ev0), "event");
  CK(cudaEventCreate(&ctx->ev1), "event");
  const int m = K->m, n = K->n;
  const int64_t nnz = K->nnz;
  cudaStream_t st = ctx->st;
  // device copies of the input (host or device pointers)
  // index and value arrays are zero-padded by kSlabNnz entries (the slab kernels
  // read whole slabs)
  int32_t *rp = dalloc<int32_t>(ctx->rp, (size_t)m + 1), *ci = dalloc<int32_t>(ctx->ci, nnz + kSlabNnz);
  double *val = dalloc<double>(ctx->val, nnz + kSlabNnz);
  double *dc = dalloc<double>(ctx->c, n), *dq = dalloc<double>(ctx->q, m), *dl = dalloc<double>(ctx->l, n),
         *du = dalloc<double>(ctx->u, n), *dylo = dalloc<double>(ctx->ylo, m);
  uint8_t *mask = dalloc<uint8_t>(ctx->mask, m);
  if (!rp || !ci || !val || !dc || !dq || !dl || !du || !dylo || !mask)
    return fail(ctx, PDLP_ERR_OOM, "input allocation failed");
  CK(cudaMemsetAsync(ci + nnz, 0, sizeof(int32_t) * kSlabNnz, st), "pad");
  CK(cudaMemsetAsync(val + nnz, 0, sizeof(double) * kSlabNnz, st), "pad");
  CK(cudaMemcpyAsync(rp, K->row_ptr, sizeof(int32_t) * ((size_t)m + 1), cudaMemcpyDefault, st), "copy row_ptr");
  if (nnz > 0) {
    CK(cudaMemcpyAsync(ci, K->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDefault, st), "copy col_idx");
    CK(cudaMemcpyAsync(val, K->val, sizeof(double) * nnz, cudaMemcpyDefault, st), "copy val");
  }
  CK(cudaMemcpyAsync(dc, c, sizeof(double) * n, cudaMemcpyDefault, st), "copy c");
  CK(cudaMemcpyAsync(dq, q, sizeof(double) * m, cudaMemcpyDefault, st), "copy q");
  CK(cudaMemcpyAsync(dl, l, sizeof(double) * n, cudaMemcpyDefault, st), "copy l");
  CK(cudaMemcpyAsync(du, u, sizeof(double) * n, cudaMemcpyDefault, st), "copy u");
  CK(cudaMemcpyAsync(mask, ineq_mask, sizeof(uint8_t) * m, cudaMemcpyDefault, st), "copy ineq_mask");
  // validation on the device
  DevBuf errbuf;
  unsigned *derr = dalloc<unsigned>(errbuf, 1);
  int32_t *rowid = dalloc<int32_t>(ctx->rowid, nnz);
  unsigned herr = 0;
  if (!derr || !rowid) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
  CK(validate(m, n, nnz, rp, ci, val, dc, dq, dl, du, rowid, derr, &herr, st), "validate");
  if (herr) return fail(ctx, PDLP_ERR_INVALID_ARG, validate_message(herr));
  CK(ylo_from_mask(m, mask, dylo, st), "ylo");
  // K^T
  int32_t *trp = dalloc<int32_t>(ctx->trp, (size_t)n + 1), *tci = dalloc<int32_t>(ctx->tci, nnz + kSlabNnz),
          *perm = dalloc<int32_t>(ctx->perm, nnz);
  double *tval = dalloc<double>(ctx->tval, nnz + kSlabNnz);
  if (!trp || !tci || !perm || !tval) return fail(ctx, PDLP_ERR_OOM, "transpose allocation failed");
  CK(cudaMemsetAsync(tci + nnz, 0, sizeof(int32_t) * kSlabNnz, st), "pad");
  CK(cudaMemsetAsync(tval + nnz, 0, sizeof(double) * kSlabNnz, st), "pad");
  {
    DevBuf tmp;
    CK(build_transpose(m, n, nnz, rp, ci, trp, tci, perm, tmp, st), "transpose");
  }
  // Section 3.5 preconditioning and transform: Ruiz is queued on st and the
  // host plans the chunk schedules meanwhile; then Pock-Chambolle (whose long
  // rows are summed on the host), the transform and the step size
  double *D1 = dalloc<double>(ctx->D1, m), *D2 = dalloc<double>(ctx->D2, n);
  double *cs = dalloc<double>(ctx->cs, n), *qs = dalloc<double>(ctx->qs, m), *ls = dalloc<double>(ctx->ls, n),
         *us = dalloc<double>(ctx->us, n), *ylos = dalloc<double>(ctx->ylos, m);
  double *i1 = dalloc<double>(ctx->D1inv, m), *i2 = dalloc<double>(ctx->D2inv, n);
  DevBuf rbuf, cbuf, mb;
  double *rb = dalloc<double>(rbuf, m), *cb = dalloc<double>(cbuf, n);
  unsigned long long *dmax = dalloc<unsigned long long>(mb, 1);
  if (!D1 || !D2 || !cs || !qs || !ls || !us || !ylos || !rb || !cb || !i1 || !i2 || !dmax)
    return fail(ctx, PDLP_ERR_OOM, "allocation failed");
  // row starts of K and K^T (final since the transpose); the long rows that
  // the preconditioning treats apart
  std::vector<int32_t> hrp((size_t)m + 1), htrp((size_t)n + 1);
  CK(cudaMemcpy(hrp.data(), rp, sizeof(int32_t) * hrp.size(), cudaMemcpyDeviceToHost), "row_ptr");
  CK(cudaMemcpy(htrp.data(), trp, sizeof(int32_t) * htrp.size(), cudaMemcpyDeviceToHost), "row_ptr");
  PrecondPlan pp;
  plan_precondition(m, hrp.data(), n, htrp.data(), pp);
  DevBuf segbuf;
  ScanSeg *dseg = pp.segK.size() + pp.segKT.size() > 0
                      ? dalloc<ScanSeg>(segbuf, pp.segK.size() + pp.segKT.size())
                      : nullptr;
  if (pp.segK.size() + pp.segKT.size() > 0) {
    if (!dseg) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
    if (!pp.segK.empty())
      CK(cudaMemcpy(dseg, pp.segK.data(), sizeof(ScanSeg) * pp.segK.size(), cudaMemcpyHostToDevice), "segments");
    if (!pp.segKT.empty())
      CK(cudaMemcpy(dseg + pp.segK.size(), pp.segKT.data(), sizeof(ScanSeg) * pp.segKT.size(),
                    cudaMemcpyHostToDevice), "segments");
  }
  CK(ruiz(m, n, nnz, rp, ci, rowid, val, trp, tval, perm, o.ruiz_iters, D1, D2, rb, cb, dseg, (int)pp.segK.size(),
          dseg ? dseg + pp.segK.size() : nullptr, (int)pp.segKT.size(), st),
     "Ruiz");
  // host planning, K and K^T on two threads: warp-chunk schedules, the
  // balanced chunk lists of the persistent kernel's warps, and (for the slab
  // engine only) the fixed-size slabs
  struct Plan {
    std::vector<Chunk> chunks;
    std::vector<LongRow> longrows;
    int32_t nseg = 0;
    std::vector<int32_t> widx, woff;
    int32_t cmax = 0;
    std::vector<int32_t> first, head, tail;
    std::vector<SplitRow> splits;
    int32_t nparts = 0;
  };
  Plan pK, pKT;
  const int nw = persist_warps(), wpc = persist_warps_per_cta();
  const bool slabs = o.persistent == 2;
  auto plan = [nw, wpc, slabs](int32_t rows, const std::vector<int32_t> &hr, Plan &pl) {
    build_schedule(rows, hr.data(), pl.chunks, pl.longrows, pl.nseg);
    if (nw > 0) assign_chunks(pl.chunks, hr.data(), nw, wpc, pl.widx, pl.woff, pl.cmax);
    if (slabs) build_slabs(rows, hr.data(), pl.first, pl.head, pl.tail, pl.splits, pl.nparts);
  };
  {
    // (no exception may cross the C ABI: without a second thread, plan both here)
    std::thread tK;
    bool threaded = true;
    try {
      tK = std::thread([&] { plan(m, hrp, pK); });
    } catch (...) {
      threaded = false;
    }
    plan(n, htrp, pKT);
    if (threaded) tK.join();
    else plan(m, hrp, pK);
  }
  if (o.pock_chambolle)
    CK(pock_chambolle(m, n, nnz, rp, ci, rowid, val, trp, tval, perm, D1, D2, rb, cb, pp, hrp.data(), htrp.data(),
                      st),
       "Pock-Chambolle");
  CK(transform(m, n, D1, D2, dc, dq, dl, du, dylo, cs, qs, ls, us, ylos, st), "transform");
  k_recip<<<std::min<int64_t>((m + 255) / 256, 1024), 256, 0, st>>>(D1, m, i1);
  k_recip<<<std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(D2, n, i2);
  CK(cudaGetLastError(), "reciprocals");
  // step size 1 / max |K~_ij| (Algorithm 1 initialisation)
  CK(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st), "memset");
  if (nnz > 0) k_absmax_bits<<<std::min<int64_t>((nnz + 255) / 256, 1024), 256, 0, st>>>(val, nnz, dmax);
  CK(cudaGetLastError(), "absmax");
  CK(cudaStreamSynchronize(st), "preconditioning");
  {
    unsigned long long hmax = 0ull;
    CK(cudaMemcpy(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost), "absmax");
    double kmax;
    memcpy(&kmax, &hmax, sizeof(kmax));
    ctx->eta0 = kmax > 0.0 ? 1.0 / kmax : 1.0;
  }
  // upload the schedules
  {
    ctx->hblocksK = std::move(pK.chunks);
    ctx->hblocksKT = std::move(pKT.chunks);
    const std::vector<LongRow> &lK = pK.longrows, &lKT = pKT.longrows;
    const int32_t segK = pK.nseg, segKT = pKT.nseg;
    ctx->nblocksK = (int32_t)((ctx->hblocksK.size() + kWarps - 1) / kWarps);
    ctx->nblocksKT = (int32_t)((ctx->hblocksKT.size() + kWarps - 1) / kWarps);
    Chunk *bK = dalloc<Chunk>(ctx->blocksK, ctx->hblocksK.size()), *bKT = dalloc<Chunk>(ctx->blocksKT, ctx->hblocksKT.size());
    LongRow *LK = dalloc<LongRow>(ctx->longK, lK.size()), *LKT = dalloc<LongRow>(ctx->longKT, lKT.size());
    double *sK = dalloc<double>(ctx->segK, 2 * (size_t)segK), *sKT = dalloc<double>(ctx->segKT, 2 * (size_t)segKT);
    // K^T: two sets of arrival counters (the persistent evaluation walks K^T twice)
    unsigned *cK = dalloc<unsigned>(ctx->segcntK, lK.size()), *cKT = dalloc<unsigned>(ctx->segcntKT, 2 * lKT.size());
    double *aK = dalloc<double>(ctx->lraccK, kLrAcc * lK.size()), *aKT = dalloc<double>(ctx->lraccKT, kLrAcc * lKT.size());
    ctx->nlongK = (int32_t)lK.size();
    ctx->nlongKT = (int32_t)lKT.size();
    ctx->nsegKT = segKT;
    if (!bK || !bKT || !LK || !LKT || !sK || !sKT || !cK || !cKT || !aK || !aKT)
      return fail(ctx, PDLP_ERR_OOM, "allocation failed");
    CK(cudaMemcpy(bK, ctx->hblocksK.data(), sizeof(Chunk) * ctx->hblocksK.size(), cudaMemcpyHostToDevice), "chunks");
    CK(cudaMemcpy(bKT, ctx->hblocksKT.data(), sizeof(Chunk) * ctx->hblocksKT.size(), cudaMemcpyHostToDevice), "chunks");
    if (!lK.empty()) CK(cudaMemcpy(LK, lK.data(), sizeof(LongRow) * lK.size(), cudaMemcpyHostToDevice), "long rows");
    if (!lKT.empty()) CK(cudaMemcpy(LKT, lKT.data(), sizeof(LongRow) * lKT.size(), cudaMemcpyHostToDevice), "long rows");
    CK(cudaMemset(cK, 0, sizeof(unsigned) * std::max<size_t>(lK.size(), 1)), "memset");
    CK(cudaMemset(cKT, 0, sizeof(unsigned) * std::max<size_t>(2 * lKT.size(), 1)), "memset");
    // fixed-size slabs (slab engine only)
    if (slabs) {
      auto up = [&](Plan &pl, DevBuf &slab, DevBuf &split, DevBuf &spart, DevBuf &scnt, DevBuf &sacc, int32_t &nslab,
                    int32_t &nsplit, int32_t &ndefer) -> int {
        nslab = (int32_t)pl.head.size();
        nsplit = (int32_t)pl.splits.size();
        ndefer = 0;
        for (const SplitRow &R : pl.splits) ndefer += split_deferred(R) ? 1 : 0;
        std::vector<int32_t> meta(pl.first);
        meta.insert(meta.end(), pl.head.begin(), pl.head.end());
        meta.insert(meta.end(), pl.tail.begin(), pl.tail.end());
        int32_t *dm = dalloc<int32_t>(slab, meta.size());
        SplitRow *ds = dalloc<SplitRow>(split, pl.splits.size());
        double *dp = dalloc<double>(spart, (size_t)pl.nparts);
        const size_t nsp = std::max<size_t>(pl.splits.size(), 1);
        unsigned *dc2 = dalloc<unsigned>(scnt, nsp);
        double *da = dalloc<double>(sacc, kLrAcc * nsp);
        if (!dm || !ds || !dp || !dc2 || !da) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
        CK(cudaMemcpy(dm, meta.data(), sizeof(int32_t) * meta.size(), cudaMemcpyHostToDevice), "slabs");
        if (!pl.splits.empty())
          CK(cudaMemcpy(ds, pl.splits.data(), sizeof(SplitRow) * pl.splits.size(), cudaMemcpyHostToDevice), "slabs");
        CK(cudaMemset(dc2, 0, sizeof(unsigned) * nsp), "memset");
        CK(cudaMemset(da, 0, sizeof(double) * kLrAcc * nsp), "memset");
        return PDLP_OK;
      };
      int rc2 = up(pK, ctx->slabK, ctx->splitK, ctx->spartK, ctx->scntK, ctx->saccK, ctx->nslabK, ctx->nsplitK,
                   ctx->ndeferK);
      if (!rc2) rc2 = up(pKT, ctx->slabKT, ctx->splitKT, ctx->spartKT, ctx->scntKT, ctx->saccKT, ctx->nslabKT,
                         ctx->nsplitKT, ctx->ndeferKT);
      if (rc2) return rc2;
    }
    // balanced chunk lists for the persistent kernel's warps
    if (nw > 0) {
      const std::vector<int32_t> &iK = pK.widx, &oK = pK.woff, &iKT = pKT.widx, &oKT = pKT.woff;
      ctx->cmaxK = pK.cmax;
      ctx->cmaxKT = pKT.cmax;
      int32_t *wK = dalloc<int32_t>(ctx->wchunkK, iK.size()), *fK = dalloc<int32_t>(ctx->woffK, oK.size());
      int32_t *wKT = dalloc<int32_t>(ctx->wchunkKT, iKT.size()), *fKT = dalloc<int32_t>(ctx->woffKT, oKT.size());
      if (!wK || !fK || !wKT || !fKT) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
      CK(cudaMemcpy(wK, iK.data(), sizeof(int32_t) * iK.size(), cudaMemcpyHostToDevice), "chunk lists");
      CK(cudaMemcpy(fK, oK.data(), sizeof(int32_t) * oK.size(), cudaMemcpyHostToDevice), "chunk lists");
      CK(cudaMemcpy(wKT, iKT.data(), sizeof(int32_t) * iKT.size(), cudaMemcpyHostToDevice), "chunk lists");
      CK(cudaMemcpy(fKT, oKT.data(), sizeof(int32_t) * oKT.size(), cudaMemcpyHostToDevice), "chunk lists");
      ctx->assign_nw = nw;
    }
  }
  double *xin = dalloc<double>(ctx->xin, n), *yin = dalloc<double>(ctx->yin, m);
  Scalars *sc = dalloc<Scalars>(ctx->scal, 1);
  if (!xin || !yin || !sc) return fail(ctx, PDLP_ERR_OOM, "allocation failed");
  CK(cudaMemsetAsync(sc, 0, sizeof(Scalars), st), "memset");
  int rc = PDLP_OK;
  if (o.unroll_T > 0) rc = setup_fp64(ctx);
  else if (o.precision == PDLP_FP64) rc = setup_fp64(ctx);
  else if (o.precision == PDLP_FP32) rc = setup_fp32(ctx);
  else rc = setup_refine(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st), "create");
  *out = hold.release();
  return PDLP_OK;
}

extern "C" int pdlp_solve(pdlp_ctx *ctx, const double *x0, const double *y0, double *x_out, double *y_out,
                          pdlp_result *res) {
  if (!ctx) return fail(nullptr, PDLP_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->pre) return solve_presolved(ctx, x0, y0, x_out, y_out, res);
  if (ctx->opts.unroll_T > 0)
    return pdlp_unroll(ctx, ctx->opts.unroll_T, ctx->opts.ckpt_every, x0, y0, x_out, y_out, nullptr);
  int rc = stage_start(ctx, x0, y0);
  if (rc) return rc;
  Scalars hs;
  pdlp_result r;
  const int prec = ctx->opts.precision;
  CK(cudaEventRecord(ctx->ev0, ctx->st), "event");
  const double *xo = nullptr, *yo = nullptr;
  if (prec == PDLP_FP64) {
    if ((rc = setup_fp64(ctx))) return rc;
    if ((rc = run_graph<double>(ctx, ctx->p64, &hs))) return rc;
    xo = ctx->p64.S.xo;
    yo = ctx->p64.S.yo;
    read_result(hs, 0.0, &r);
    r.engine = engine_of(ctx->p64);
  } else if (prec == PDLP_FP32) {
    if ((rc = setup_fp32(ctx))) return rc;
    if ((rc = run_graph<float>(ctx, ctx->p32, &hs))) return rc;
    xo = ctx->p32.S.xo;
    yo = ctx->p32.S.yo;
    read_result(hs, 0.0, &r);
    r.engine = engine_of(ctx->p32);
  } else {
    if ((rc = setup_refine(ctx))) return rc;
    RefineOutcome ro;
    auto run_inner = [ctx](Scalars *h) -> cudaError_t {
      return run_graph<float>(ctx, ctx->pc32, h) == PDLP_OK ? cudaSuccess : cudaErrorUnknown;
    };
    RefineLimits lim;
    lim.iter_limit = ctx->opts.iter_limit;
    lim.kkt_limit = ctx->opts.kkt_pass_limit;
    lim.time_limit_s = ctx->opts.time_limit_s;
    double *xi = reinterpret_cast<double *>(ctx->xin.ptr()), *yi = reinterpret_cast<double *>(ctx->yin.ptr());
    cudaError_t e = refine_solve(ctx->ref, ctx->p64.K, ctx->p64.KT, ctx->p64.P, ctx->pc32.S, run_inner,
                                 ctx->opts.rel_tol, ctx->opts.inner_tol, ctx->opts.refine_rounds, lim, xi, yi,
                                 ctx->st, &ro);
    if (e) return cuda_fail(ctx, e, "refinement");
    xo = ro.x;
    yo = ro.y;
    memset(&r, 0, sizeof(r));
    r.status = ro.status;
    r.iters = ro.iters;
    r.kkt_passes = ro.kkt_passes;
    r.restarts = ro.restarts;
    r.refine_rounds = ro.rounds;
    r.engine = engine_of(ctx->pc32);
    r.primal_obj = ro.kkt[0];
    r.dual_obj = ro.kkt[1];
    r.gap = ro.kkt[2];
    r.pres = ro.kkt[3];
    r.dres = ro.kkt[4];
    r.rel_gap = ro.kkt[5];
    r.rel_pres = ro.kkt[6];
    r.rel_dres = ro.kkt[7];
    int spent = 0;
    if (ro.finish) {
      // the float32 corrections stopped paying: float64 PDLP from the refined
      // point (staged as the start point) with what is left of the budget
      if (refine_set_limits(ctx->ref, lim, ro.iters, ro.kkt_passes, ro.seconds, ctx->st, &spent, &e)) {
        CK(cudaMemcpyAsync(xi, ro.x, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->st), "finish x0");
        CK(cudaMemcpyAsync(yi, ro.y, sizeof(double) * ctx->m, cudaMemcpyDeviceToDevice, ctx->st), "finish y0");
        if ((rc = run_graph<double>(ctx, ctx->p64, &hs))) return rc;
        pdlp_result rf;
        read_result(hs, 0.0, &rf);
        const double e_ref = fmax(r.rel_gap, fmax(r.rel_pres, r.rel_dres));
        const double e_fin = fmax(rf.rel_gap, fmax(rf.rel_pres, rf.rel_dres));
        if (rf.status == kOptimal || e_fin <= e_ref) {
          r = rf;
          r.engine = engine_of(ctx->p64);
          xo = ctx->p64.S.xo;
          yo = ctx->p64.S.yo;
        } else {
          r.status = rf.status;  // the finish ended at a limit further from Eq. (15): keep the refined point
        }
        r.iters = ro.iters + hs.k;
        r.kkt_passes = ro.kkt_passes + hs.attempts;
        r.restarts = ro.restarts + hs.restarts;
        r.refine_rounds = ro.rounds;
        r.finish_iters = hs.k;
      } else {
        if (e) return cuda_fail(ctx, e, "refinement limits");
        r.status = spent;
      }
    }
  }
  CK(cudaEventRecord(ctx->ev1, ctx->st), "event");
  if (x_out) CK(cudaMemcpyAsync(x_out, xo, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st), "x_out");
  if (y_out) CK(cudaMemcpyAsync(y_out, yo, sizeof(double) * ctx->m, cudaMemcpyDefault, ctx->st), "y_out");
  CK(cudaStreamSynchronize(ctx->st), "solve");
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "event");
  r.seconds = ms * 1e-3;
  if (res) *res = r;
  return PDLP_OK;
}

extern "C" int pdlp_get_scaled(pdlp_ctx *ctx, double *Kval, int32_t *KT_row_ptr, int32_t *KT_col_idx,
                               double *KTval, int32_t *KT_perm, double *D1, double *D2, double *cs,
                               double *qs, double *ls, double *us) {
  if (!ctx) return fail(nullptr, PDLP_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->pre) return fail(ctx, PDLP_ERR_STATE, "pdlp_get_scaled: not available on a presolved context");
  const size_t n = ctx->n, m = ctx->m, nnz = ctx->nnz;
  cudaStream_t st = ctx->st;
  auto cp = [&](void *dst, const DevBuf &src, size_t bytes) -> cudaError_t {
    if (!dst || bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src.ptr(), bytes, cudaMemcpyDefault, st);
  };
  CK(cp(Kval, ctx->val, 8 * nnz), "copy");
  CK(cp(KT_row_ptr, ctx->trp, 4 * (n + 1)), "copy");
  CK(cp(KT_col_idx, ctx->tci, 4 * nnz), "copy");
  CK(cp(KTval, ctx->tval, 8 * nnz), "copy");
  CK(cp(KT_perm, ctx->perm, 4 * nnz), "copy");
  CK(cp(D1, ctx->D1, 8 * m), "copy");
  CK(cp(D2, ctx->D2, 8 * n), "copy");
  CK(cp(cs, ctx->cs, 8 * n), "copy");
  CK(cp(qs, ctx->qs, 8 * m), "copy");
  CK(cp(ls, ctx->ls, 8 * n), "copy");
  CK(cp(us, ctx->us, 8 * n), "copy");
  CK(cudaStreamSynchronize(st), "copy");
  return PDLP_OK;
}

extern "C" int pdlp_normalized_gap(pdlp_ctx *ctx, const double *x, const double *y, double omega, double r,
                                   double *mu, double *value) {
  if (!ctx || !x || !y) return fail(ctx, PDLP_ERR_INVALID_ARG, "NULL argument");
  if (ctx->pre) return fail(ctx, PDLP_ERR_STATE, "pdlp_normalized_gap: not available on a presolved context");
  if (!(r > 0.0) || !(omega > 0.0)) return fail(ctx, PDLP_ERR_INVALID_ARG, "r and omega must be > 0");
  int rc = setup_fp64(ctx);
  if (rc) return rc;
  Precision<double> &pr = ctx->p64;
  State<double> &S = pr.S;
  cudaStream_t st = ctx->st;
  CK(cudaMemcpyAsync(S.x[0], x, sizeof(double) * ctx->n, cudaMemcpyDefault, st), "x");
  CK(cudaMemcpyAsync(S.y[0], y, sizeof(double) * ctx->m, cudaMemcpyDefault, st), "y");
  launch_spmv<double>(pr.KT, S.y[0], S.KTy_cur, st);
  launch_spmv<double>(pr.K, S.x[0], S.Kx[0], st);
  CK(cudaGetLastError(), "spmv");
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st), "scalars");
  CK(cudaStreamSynchronize(st), "sync");
  hs.cur = 0;
  hs.do_gap = 1;
  hs.restart = 0;
  for (int a = 0; a < kGapSlots; ++a) {
    hs.g_active[a] = 0;
    hs.mu[a] = INFINITY;
  }
  hs.g_active[0] = 1;
  hs.g_r2[0] = r * r;
  hs.g_omega[0] = omega;
  hs.g_inv_omega[0] = 1.0 / omega;
  hs.g_W[0] = hs.g_V[0] = hs.g_A[0] = 0.0;
  hs.g_prefix[0] = 0u;
  CK(cudaMemcpyAsync(S.s, &hs, sizeof(Scalars), cudaMemcpyHostToDevice, st), "scalars");
  CK(launch_gap_slots<double>(pr.P, S, 0, 1, 0, 152, st), "gap");
  CK(cudaMemcpyAsync(&hs, S.s, sizeof(Scalars), cudaMemcpyDeviceToHost, st), "scalars");
  CK(cudaStreamSynchronize(st), "sync");
  if (mu) *mu = hs.mu[0];
  if (value) *value = hs.gval[0];
  return PDLP_OK;
}

extern "C" int pdlp_get_trace(pdlp_ctx *ctx, double *out, int32_t max_records, int32_t *count) {
  if (!ctx) return fail(nullptr, PDLP_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->pre) {
    if (!ctx->inner) return fail(ctx, PDLP_ERR_STATE, "the presolve decided the LP: nothing was iterated");
    const int rc = pdlp_get_trace(ctx->inner, out, max_records, count);
    return rc ? fail(ctx, rc, pdlp_last_error(ctx->inner)) : rc;
  }
  const double *tr = nullptr;
  if (ctx->opts.precision == PDLP_FP64 && ctx->p64.ready) tr = ctx->p64.S.trace;
  else if (ctx->opts.precision == PDLP_FP32 && ctx->p32.ready) tr = ctx->p32.S.trace;
  else if (ctx->pc32.ready) tr = ctx->pc32.S.trace;
  else if (ctx->p64.ready) tr = ctx->p64.S.trace;
  if (!tr) return fail(ctx, PDLP_ERR_STATE, "no solve has run on this context");
  Scalars hs;
  CK(cudaMemcpy(&hs, ctx->scal.ptr(), sizeof(Scalars), cudaMemcpyDeviceToHost), "trace");
  const int total = hs.trace_n;
  const int avail = total < kTraceCap ? total : kTraceCap;
  const int take = max_records < avail ? max_records : avail;
  if (count) *count = total;
  // oldest record first: the ring from its oldest slot to the end, then from slot 0
  const int first = (total - avail) % kTraceCap;
  const int n1 = take < kTraceCap - first ? take : kTraceCap - first;
  if (n1 > 0)
    CK(cudaMemcpy(out, tr + (size_t)first * kTraceLen, sizeof(double) * kTraceLen * (size_t)n1,
                  cudaMemcpyDeviceToHost), "trace");
  if (take > n1)
    CK(cudaMemcpy(out + (size_t)n1 * kTraceLen, tr, sizeof(double) * kTraceLen * (size_t)(take - n1),
                  cudaMemcpyDeviceToHost), "trace");
  return PDLP_OK;
}

extern "C" int pdlp_time_step_kernels(pdlp_ctx *ctx, int32_t reps, float *ms) {
  if (!ctx || !ms || reps < 1) return fail(ctx, PDLP_ERR_INVALID_ARG, "bad argument");
  if (ctx->pre) {
    if (!ctx->inner) return fail(ctx, PDLP_ERR_STATE, "the presolve decided the LP: nothing was iterated");
    const int rc = pdlp_time_step_kernels(ctx->inner, reps, ms);
    return rc ? fail(ctx, rc, pdlp_last_error(ctx->inner)) : rc;
  }
  cudaError_t e;
  const int prec = ctx->opts.precision;
  if (prec == PDLP_FP64 && ctx->p64.ready)
    e = time_step_kernels<double>(ctx->p64.K, ctx->p64.KT, ctx->p64.P, ctx->p64.S, reps, ctx->st, ms, ms + 1);
  else if (prec == PDLP_FP32 && ctx->p32.ready)
    e = time_step_kernels<float>(ctx->p32.K, ctx->p32.KT, ctx->p32.P, ctx->p32.S, reps, ctx->st, ms, ms + 1);
  else if (prec == PDLP_FP32_REFINE && ctx->pc32.ready)
    e = time_step_kernels<float>(ctx->pc32.K, ctx->pc32.KT, ctx->pc32.P, ctx->pc32.S, reps, ctx->st, ms, ms + 1);
  else
    return fail(ctx, PDLP_ERR_STATE, "no solver state for the context's precision");
  if (e) return cuda_fail(ctx, e, "time_step_kernels");
  ms[2] = 0.f;
  if (prec == PDLP_FP64 && ctx->p64.pg.grid > 0)
    e = time_persist<double>(ctx->p64.K, ctx->p64.KT, ctx->p64.P, ctx->p64.S, ctx->p64.pg, reps, ctx->st, ms + 2);
  else if (prec == PDLP_FP32 && ctx->p32.pg.grid > 0)
    e = time_persist<float>(ctx->p32.K, ctx->p32.KT, ctx->p32.P, ctx->p32.S, ctx->p32.pg, reps, ctx->st, ms + 2);
  else if (prec == PDLP_FP32_REFINE && ctx->pc32.pg.grid > 0)
    e = time_persist<float>(ctx->pc32.K, ctx->pc32.KT, ctx->pc32.P, ctx->pc32.S, ctx->pc32.pg, reps, ctx->st,
                            ms + 2);
  if (e) return cuda_fail(ctx, e, "time_persist");
  ms[3] = 0.f;
  if (prec == PDLP_FP64 && ctx->p64.pe.grid > 0)
    e = time_eval_persist<double>(ctx->p64.K, ctx->p64.KT, ctx->p64.KTb, ctx->p64.P, ctx->p64.S, ctx->p64.pe, reps,
                                  ctx->st, ms + 3);
  if (e) return cuda_fail(ctx, e, "time_eval_persist");
  return PDLP_OK;
}

extern "C" const char *pdlp_last_error(const pdlp_ctx *ctx) {
  if (ctx && !ctx->err.empty()) return ctx->err.c_str();
  return g_last_error.c_str();
}

extern "C" void pdlp_destroy(pdlp_ctx *ctx) { delete ctx; }

// Unrolled map and its adjoint (unroll.cu)
extern "C" int pdlp_unroll(pdlp_ctx *ctx, int32_t T, int32_t ckpt_every, const double *x0, const double *y0,
                           double *x_out, double *y_out, double *eta_out) {
  if (!ctx) return fail(nullptr, PDLP_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->pre) return fail(ctx, PDLP_ERR_STATE, "pdlp_unroll: not available on a presolved context");
  if (T < 1 || ckpt_every < 1 || ckpt_every > kMaxEval)
    return fail(ctx, PDLP_ERR_INVALID_ARG, "need T >= 1 and 1 <= ckpt_every <= 256");
  const bool f32 = ctx->opts.precision == PDLP_FP32;
  int rc = setup_fp64(ctx);  // float64 K~ for the adjoint
  if (!rc && f32) rc = setup_fp32(ctx);
  if (rc) return rc;
  rc = stage_start(ctx, x0, y0);
  if (rc) return rc;
  UnrollBuffers &U = ctx->unr;
  U.nnz = ctx->nnz;
  U.row = reinterpret_cast<const int32_t *>(ctx->rowid.ptr());
  const double *xin = reinterpret_cast<const double *>(ctx->xin.ptr());
  const double *yin = reinterpret_cast<const double *>(ctx->yin.ptr());
  cudaError_t e;
  if (f32) {
    Precision<float> &pr = ctx->p32;
    e = unroll_forward<float>(U, pr.K, pr.KT, pr.P, pr.S, pr.pg, pr.init, ctx->opts.primal_importance,
                              pr.normpart_ptr, T, ckpt_every, xin, yin, ctx->st);
  } else {
    Precision<double> &pr = ctx->p64;
    e = unroll_forward<double>(U, pr.K, pr.KT, pr.P, pr.S, pr.pg, pr.init, ctx->opts.primal_importance,
                               pr.normpart_ptr, T, ckpt_every, xin, yin, ctx->st);
  }
  if (e) return cuda_fail(ctx, e, "unroll");
  if (U.status == kWaitTimeout)
    return fail(ctx, PDLP_ERR_TIMEOUT, "a grid-wide barrier of the persistent step kernel timed out");
  if (!U.ready)
    return fail(ctx, PDLP_ERR_STATE, U.status == kNumErr ? "unrolled map stopped: numerical error"
                                                         : "unrolled map stopped: attempt limit");
  if (x_out) CK(cudaMemcpyAsync(x_out, U.xo, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st), "x_out");
  if (y_out) CK(cudaMemcpyAsync(y_out, U.yo, sizeof(double) * ctx->m, cudaMemcpyDefault, ctx->st), "y_out");
  if (eta_out) CK(cudaMemcpyAsync(eta_out, U.eta, sizeof(double) * T, cudaMemcpyDefault, ctx->st), "eta");
  CK(cudaStreamSynchronize(ctx->st), "unroll");
  return PDLP_OK;
}

extern "C" int pdlp_grad(pdlp_ctx *ctx, const double *dL_dx, const double *dL_dy, double *dc, double *dq,
                         double *dK_val) {
  if (!ctx || !dL_dx) return fail(ctx, PDLP_ERR_INVALID_ARG, "NULL argument");
  if (ctx->pre) return fail(ctx, PDLP_ERR_STATE, "pdlp_grad: not available on a presolved context");
  if (!ctx->unr.ready) return fail(ctx, PDLP_ERR_STATE, "pdlp_grad needs a preceding unrolled solve");
  cudaError_t e =
      ctx->unr.fp32 ? unroll_backward<float>(ctx->unr, ctx->p32.K, ctx->p32.KT, ctx->p32.P, ctx->p64.K, ctx->p64.KT,
                                             ctx->p64.P, dL_dx, dL_dy, ctx->st)
                    : unroll_backward<double>(ctx->unr, ctx->p64.K, ctx->p64.KT, ctx->p64.P, ctx->p64.K,
                                              ctx->p64.KT, ctx->p64.P, dL_dx, dL_dy, ctx->st);
  if (e) return cuda_fail(ctx, e, "grad");
  if (dc) CK(cudaMemcpyAsync(dc, ctx->unr.dc, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st), "dc");
  if (dq) CK(cudaMemcpyAsync(dq, ctx->unr.dq, sizeof(double) * ctx->m, cudaMemcpyDefault, ctx->st), "dq");
  if (dK_val) CK(cudaMemcpyAsync(dK_val, ctx->unr.dK, sizeof(double) * ctx->nnz, cudaMemcpyDefault, ctx->st), "dK");
  CK(cudaStreamSynchronize(ctx->st), "grad");
  return PDLP_OK;
}
