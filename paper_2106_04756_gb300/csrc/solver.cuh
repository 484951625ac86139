// Launchers of the iteration kernels (solver.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace pdlp {

// Per-solve settings written into Scalars by k_init_scalars.
struct ScalarInit {
  double eta0, rel_tol, beta_suff, beta_nec, beta_art, pw_theta, eps_zero;
  long long iter_limit, attempt_limit;
  unsigned long long time_limit_ns;
  unsigned long long wait_ns;  // bound of device-side waits (grid barriers)
  int wait_extra;              // 1: the first barrier of a persistent launch cannot complete (timeout test)
  int eval_every, adaptive_restart, pw_update, const_step;
  double omega0;  // > 0: initial primal weight instead of InitializePrimalWeight
  int restart_to_current;  // 0: restart candidate always the average (Appendix C.2)
  int mp;                  // 1: Malitsky-Pock line search (Appendix C.1)
  double mp_breaking, mp_downscaling, mp_interpolation;
  const double *tol_dev;  // non-null: read rel_tol from this device double at each solve
  const long long *lim_dev;  // non-null: iter_limit, attempt_limit, time_limit_ns (0: none) read
                             // from these three device values at each solve
  int stall_evals;        // > 0: stop (kStalled) after this many evaluations without a 10% gain
};

template <typename T> cudaError_t set_kernel_attributes();
template <typename T>
cudaError_t launch_gap_slots(const Problem<T> &P, const State<T> &S, int s_begin, int s_end, int when_restart,
                             int grid, cudaStream_t st);
template <typename T>
cudaError_t time_step_kernels(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                              int reps, cudaStream_t st, float *ms_primal, float *ms_dual);
template <typename T> void launch_spmv(const Mat<T> &A, const T *v, T *out, cudaStream_t st);
// ||A||_2 by power iteration on A^T A (A = K with its transpose AT): `iters`
// steps from v = 1/sqrt(n); scratch v (n), w (m), u (n) and 2 doubles.
template <typename T>
cudaError_t power_norm(const Mat<T> &A, const Mat<T> &AT, int iters, T *v, T *w, T *u, double *nrm,
                       cudaStream_t st, double *out);
// CTAs of the slab kernels' launches (K.slab_grid, KT.slab_grid).
template <typename T> cudaError_t plan_slab_grid(Mat<T> &K, Mat<T> &KT);
// One step attempt (k_primal, k_dual with the step test) outside any graph.
template <typename T>
cudaError_t launch_step_pair(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                             cudaStream_t st);
template <typename T>
void launch_problem_norms(const Problem<T> &P, Scalars *s, double primal_importance, double *part, int grid,
                          cudaStream_t st);
template <typename T>
void launch_init(const Problem<T> &P, const State<T> &S, const Mat<T> &K, const ScalarInit &in,
                 const double *x0, const double *y0, cudaStream_t st);
template <typename T>
void launch_eval(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S, cudaStream_t st);
template <typename T> void launch_output(const Problem<T> &P, const State<T> &S, cudaStream_t st);
template <typename T>
cudaError_t build_solve_graph(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                              const State<T> &S, const ScalarInit &in, double primal_importance, double *norm_part,
                              const double *x0_dev, const double *y0_dev, int gap_grid, const PersistGeo &pg,
                              const PersistGeo &pe,
                              cudaStream_t st, cudaStream_t st2, cudaStream_t st3, cudaStream_t st4,
                              cudaGraphExec_t *exec);
// Persistent step kernel (persistent.cu).  mode 0: off.  Leaves pg->grid = 0
// when the kernel's layout does not fit or no chunk assignment exists for
// its grid (assign_nw warps).  cmax_*: most chunks of one warp.
int persist_warps();  // warps of the persistent grid on the current device (0 on error)
int persist_warps_per_cta();
template <typename T>
cudaError_t persist_plan(int cmax_kt, int cmax_k, int assign_nw, int mode, int l1_gather, PersistGeo *pg);
template <typename T>
cudaError_t launch_persist(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                           const PersistGeo &pg, cudaStream_t st);
template <typename T>
cudaError_t time_persist(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                         const PersistGeo &pg, int reps, cudaStream_t st, float *ms_attempt);
// Persistent evaluation kernel (persistent.cu): the evaluation's products and
// Eq. (15) terms on the step kernel's grid; float64 contexts only
// (pe->grid = 0 otherwise, and the separate evaluation kernels run).
template <typename T>
cudaError_t eval_plan(const PersistGeo &pg, int cmax_kt, int cmax_k, PersistGeo *pe);
template <typename T>
cudaError_t launch_eval_persist(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                                const State<T> &S, const PersistGeo &pe, cudaStream_t st);
template <typename T>
cudaError_t time_eval_persist(const Mat<T> &K, const Mat<T> &KT, const Mat<T> &KTb, const Problem<T> &P,
                              const State<T> &S, const PersistGeo &pe, int reps, cudaStream_t st, float *ms);

template <typename T>
cudaError_t run_stepped(const Mat<T> &K, const Mat<T> &KT, const Problem<T> &P, const State<T> &S,
                        const ScalarInit &in, double primal_importance, double *norm_part, const double *x0_dev,
                        const double *y0_dev, int gap_grid, const PersistGeo &pg, cudaStream_t st, Scalars *host);

}  // namespace pdlp
