// Unrolled PDHG and its adjoint (unroll.cu).
#pragma once

#include "common.cuh"
#include "prep.cuh"

namespace pdlp {

struct UnrollBuffers {
  bool ready = false;
  int32_t T = 0, ckpt = 0;
  double omega = 1.0;
  DevBuf vec, ckpts, grads, etab, parts;
  double *xo = nullptr, *yo = nullptr, *eta = nullptr;
  double *dc = nullptr, *dq = nullptr, *dK = nullptr;
};

cudaError_t unroll_forward(UnrollBuffers &U, const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                           double eta0, double eps_zero, int32_t T, int32_t ckpt_every, const double *x0,
                           const double *y0, cudaStream_t st);
cudaError_t unroll_backward(UnrollBuffers &U, const Mat<double> &K, const Mat<double> &KT, const Problem<double> &P,
                            const int32_t *perm, const double *dL_dx, const double *dL_dy, cudaStream_t st);

}  // namespace pdlp
