// Presolve-lite and postsolve (presolve.cu).
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "prep.cuh"

namespace pdlp {

// Outcome codes of the presolve (besides the solver statuses).
enum : int { kPreReduced = 0, kPrimalInfeasible = 7, kDualInfeasible = 8 };

// A presolved LP: the original problem (device copies and its K^T), the maps
// between original and reduced rows / columns, the values of the removed
// columns, and the reduced problem handed to the solver.
struct Presolve {
  int32_t m0 = 0, n0 = 0;
  int64_t nnz0 = 0;
  int32_t m1 = 0, n1 = 0;
  int64_t nnz1 = 0;
  int status = kPreReduced;  // kPreReduced, kOptimal (nothing left), kPrimalInfeasible, kDualInfeasible
  double qnorm = 0.0, cnorm = 0.0;  // ||q||_2, ||c||_2 of the original problem
  DevBuf rp0, ci0, val0, c0, q0, l0, u0, ineq0, rowid0;  // original problem
  DevBuf trp0, tci0, tval0, tperm0, ttmp;                // its K^T
  DevBuf rownew, colnew, xfix, qsh, cnt, flags;          // maps, removed values, shifted q
  DevBuf rp1, ci1, val1, c1, q1, l1, u1, ineq1;          // reduced problem
  DevBuf x1, y1, kx, kty, part;                          // solve / evaluation scratch
};

// Runs the presolve on the validated original problem already copied into
// pre (rp0 ... ineq0, rowid0): fixed variables (l_j = u_j) are substituted,
// rows left without nonzeros are dropped (or report primal infeasibility),
// columns without nonzeros are set at their optimal bound (or report an
// unbounded LP), and the rest is compacted into rp1 ... ineq1.
cudaError_t presolve_run(Presolve &pre, cudaStream_t st);

// Maps a start point of the original problem to the reduced one (device
// buffers pre.x1, pre.y1; zero where the input pointer is null).
cudaError_t presolve_map_start(Presolve &pre, const double *x0, const double *y0, cudaStream_t st);

// Expands a reduced solution (x1, y1: device, or null when nothing was
// left) to the original problem (x, y: device) and evaluates Eq. (15) there:
// kkt = [primal obj, dual obj, gap, ||pres||, ||dres||, rel gap, rel pres, rel dres].
cudaError_t postsolve(Presolve &pre, const double *x1, const double *y1, double *x, double *y, double *kkt,
                      cudaStream_t st);

}  // namespace pdlp
