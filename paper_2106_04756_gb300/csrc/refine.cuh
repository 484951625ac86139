// Float32 inner solves inside a float64 iterative-refinement loop (refine.cu).
#pragma once

#include <functional>

#include "common.cuh"
#include "prep.cuh"

namespace pdlp {

// Device pointers of the refinement state (passed to kernels by value).
struct RefView {
  // current point (original space) and its scaled copy / products
  double *xh, *yh, *xt, *yt, *Kx, *KTy;
  double *xb, *yb;  // best point so far (restored if a round makes Eq. (15) worse)
  // correction LP, original space (float64) and preconditioned (float32)
  double *c, *q, *l, *u, *ylo;
  float *cs, *qs, *ls, *us, *ylos;
  double *partc;
  unsigned *ticket;
  double *rsc;  // [0..4] Eq. (15) terms at (xh, yh), [8] primal violation, [9] dual violation
};

struct RefineBuffers {
  bool ready = false;
  int32_t m = 0, n = 0, nbK = 0, nbKT = 0;
  DevBuf vec;    // float64 vectors
  DevBuf vec32;  // float32 correction data
  DevBuf part, rs;
  DevBuf tol;    // Eq. (15) tolerance of the next inner solve (read by its k_init_scalars)
  DevBuf lim;    // iteration, KKT-pass and time (ns) limits of the next solve (float32 or the
                 // float64 finish), read by its k_init_scalars
  RefView v{};
};

// Budget of one PDLP_FP32_REFINE solve: the caller's limits, shared by every
// inner solve and the float64 finish.
struct RefineLimits {
  long long iter_limit = 0, kkt_limit = 0;
  double time_limit_s = 0.0;  // <= 0: none
};

struct RefineOutcome {
  int status = 0, rounds = 0;
  // the float32 rounds stopped gaining (a round gained less than
  // kRefineMinGain, made Eq. (15) worse, or the round cap was reached) with
  // budget left: the caller finishes with float64 PDLP from (x, y)
  bool finish = false;
  double seconds = 0.0;  // host time spent in the loop (for the finish's time budget)
  long long iters = 0, kkt_passes = 0, restarts = 0;
  double kkt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double *x = nullptr, *y = nullptr;  // device, original space
};

cudaError_t refine_alloc(RefineBuffers &R, int32_t m, int32_t n, int32_t nbK, int32_t nbKT);
// Device limits of the next solve (R.lim, allocated on first use): what is
// left of `L` after `iters`, `passes` and `secs`.  Returns 0 with the limit's
// status in *spent when nothing is left, else 1.
int refine_set_limits(RefineBuffers &R, const RefineLimits &L, long long iters, long long passes, double secs,
                      cudaStream_t st, int *spent, cudaError_t *err);
long long *refine_limits_dev(RefineBuffers &R);
Problem<float> refine_problem(RefineBuffers &R, const Problem<double> &P64);



// run_inner runs one float32 solve of the correction problem held in R (start
// point: the staging buffers) to the tolerance in R.tol and returns its final
// scalars in *hs (host).
cudaError_t refine_solve(RefineBuffers &R, const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                         const State<float> &Sc, const std::function<cudaError_t(Scalars *)> &run_inner,
                         double tol, double inner_tol, int max_rounds, const RefineLimits &lim,
                         const double *x_stage, const double *y_stage, cudaStream_t st, RefineOutcome *out);

}  // namespace pdlp
