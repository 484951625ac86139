// Create-time routines (prep.cu) and a small owning device buffer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace pdlp {

// Owning device allocation (cudaMalloc / cudaFree); get() reallocates on growth.
class DevBuf {
 public:
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { reset(); }
  void *get(size_t bytes) {
    if (bytes <= cap_ && p_) return p_;
    reset();
    if (cudaMalloc(&p_, bytes ? bytes : 1) != cudaSuccess) { p_ = nullptr; cap_ = 0; return nullptr; }
    cap_ = bytes;
    return p_;
  }
  void reset() {
    if (p_) cudaFree(p_);
    p_ = nullptr;
    cap_ = 0;
  }
  void *ptr() const { return p_; }

 private:
  void *p_ = nullptr;
  size_t cap_ = 0;
};

const char *validate_message(unsigned bits);
// Checks the input (row_ptr, column range and order, finite data, bounds);
// on a valid row_ptr also fills rowid[nnz] with the row of every nonzero.
cudaError_t validate(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                     const double *val, const double *c, const double *q, const double *l,
                     const double *u, int32_t *rowid, unsigned *derr, unsigned *herr, cudaStream_t st);
cudaError_t exclusive_scan(const int *in, int64_t n, int *out, int *total, int *tmp, cudaStream_t st);
int64_t scan_tmp_ints(int64_t n);
cudaError_t build_transpose(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                            int32_t *trp, int32_t *tci, int32_t *perm, DevBuf &tmp, cudaStream_t st);
// Section 3.5 preconditioning in two calls, with the long rows of a
// PrecondPlan (schedule.h) handled apart.
// Ruiz equilibration (Section 3.5, ruiz_iters passes), queued on st: D1, D2
// from 1, val / tval scaled in place; dsegK / dsegKT: the plan's segments on
// the device.
cudaError_t ruiz(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci, const int32_t *rowid,
                 double *val, const int32_t *trp, double *tval, const int32_t *perm, int ruiz_iters, double *D1,
                 double *D2, double *rbuf, double *cbuf, const ScanSeg *dsegK, int nsegK, const ScanSeg *dsegKT,
                 int nsegKT, cudaStream_t st);
// Pock-Chambolle alpha = 1 (Section 3.5) after ruiz(); waits for st when the
// plan has long rows (their sums are taken on the host).
cudaError_t pock_chambolle(int32_t m, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                           const int32_t *rowid, double *val, const int32_t *trp, double *tval,
                           const int32_t *perm, double *D1, double *D2, double *rbuf, double *cbuf,
                           const PrecondPlan &pp, const int32_t *hrp, const int32_t *htrp, cudaStream_t st);
cudaError_t transform(int32_t m, int32_t n, const double *D1, const double *D2, const double *c,
                      const double *q, const double *l, const double *u, const double *ylo,
                      double *cs, double *qs, double *ls, double *us, double *ylos, cudaStream_t st);
cudaError_t ylo_from_mask(int32_t m, const uint8_t *ineq, double *ylo, cudaStream_t st);
cudaError_t to_float(const double *src, int64_t n, float *dst, cudaStream_t st);

}  // namespace pdlp
