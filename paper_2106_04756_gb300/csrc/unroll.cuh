// Unrolled PDHG and its adjoint (unroll.cu).
#pragma once

#include "common.cuh"
#include "prep.cuh"
#include "solver.cuh"

#include <vector>

namespace pdlp {

// State of the last unrolled map of a context: the recorded step sizes, the
// fixed primal weight, the iterates at the start of every segment of `ckpt`
// steps, the returned point and the gradient outputs.
struct UnrollBuffers {
  bool ready = false;
  int32_t T = 0, ckpt = 0, nseg = 0;
  int32_t status = 0;  // kOptimal: the map ran to T steps; else why it stopped
  bool fp32 = false;   // forward map in float32 (adjoint in float64)
  int64_t nnz = 0;
  const int32_t *row = nullptr;  // row of every nonzero of K (the context's)
  double omega = 1.0, inv_omega = 1.0;
  DevBuf ckpts, etab, outs, seg, work, fwork, grads;
  std::vector<double> eta_host;
  double *eta = nullptr, *xo = nullptr, *yo = nullptr;
  double *dc = nullptr, *dq = nullptr, *dK = nullptr;
};

// Runs T accepted steps of Algorithm 2 (fixed omega, no restarts) from
// (x0, y0) (device, original space) on the state S of arithmetic type F,
// recording the step sizes and a checkpoint every ckpt steps; xo, yo receive
// x_T, y_T.
template <typename F>
cudaError_t unroll_forward(UnrollBuffers &U, const Mat<F> &K, const Mat<F> &KT, const Problem<F> &P,
                           const State<F> &S, const PersistGeo &pg, const ScalarInit &in, double primal_importance,
                           double *norm_part, int32_t T, int32_t ckpt, const double *x0, const double *y0,
                           cudaStream_t st);

// Vector-Jacobian product of the last unrolled map: dL/dx_T (n), dL/dy_T (m,
// nullable), host or device; writes U.dc, U.dq, U.dK (original space).  The
// segments are recomputed in type F (Kf, KTf, Pf); the adjoint runs in
// float64 (K, KT, P).
template <typename F>
cudaError_t unroll_backward(UnrollBuffers &U, const Mat<F> &Kf, const Mat<F> &KTf, const Problem<F> &Pf,
                            const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                            const double *dL_dx, const double *dL_dy, cudaStream_t st);

}  // namespace pdlp
