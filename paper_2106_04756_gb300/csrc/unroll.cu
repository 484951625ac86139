// Unrolled PDHG for differentiation (filled in with the adjoint kernels).
#include "unroll.cuh"

namespace pdlp {

cudaError_t unroll_forward(UnrollBuffers &, const Mat<double> &, const Mat<double> &, const Problem<double> &,
                           double, double, int32_t, int32_t, const double *, const double *, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t unroll_backward(UnrollBuffers &, const Mat<double> &, const Mat<double> &, const Problem<double> &,
                            const int32_t *, const double *, const double *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace pdlp
