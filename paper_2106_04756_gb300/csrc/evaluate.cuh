// End of an evaluation of Eq. (15), shared by the evaluation kernels of
// solver.cu and the persistent evaluation kernel of persistent.cu.
#pragma once

#include "common.cuh"

namespace pdlp {

static __device__ __forceinline__ bool time_up(const Scalars *s) {
  return s->time_limit_ns != 0ull && global_timer_ns() - s->t0_ns > s->time_limit_ns;
}

// Finalisation of one evaluation, by every thread of the CTA that finishes
// it; ecr holds the column terms [8] then the row terms [8] (shared memory).
// Float64 square roots and divisions take hundreds of cycles each on this
// part, so each candidate's terms are split over threads of distinct warps
// (thread 0 of warp 4 c + part), and the restart radius and 1 / sum_eta are
// computed beside them; thread 0 then takes the decisions.
static __device__ void eval_finish(Scalars *s, const double *ecr, double *trace) {
  __shared__ double s_pre[3];  // r^2 of both candidates under the current omega, 1 / sum_eta
  const bool avg = s->sum_eta > 0.0;
  const double *ec = ecr, *er = ecr + 8;
  if ((threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < 8) {
    const int c = threadIdx.x >> 7, part = (threadIdx.x >> 5) & 3;
    if (!(c == 1 && !avg)) {
      double *k = s->kkt[c];
      if (part == 0) {
        const double pobj = ec[4 * c + 0] + er[4 * c + 3];
        const double dobj = ec[4 * c + 2] + er[4 * c + 1];
        const double gap = fabs(dobj - pobj);
        k[0] = pobj;
        k[1] = dobj;
        k[2] = gap;
        k[5] = gap / (1.0 + fabs(dobj) + fabs(pobj));
      } else if (part == 1) {
        const double pres = sqrt(er[4 * c + 0]);
        k[3] = pres;
        k[6] = pres / (1.0 + s->qnorm);
      } else if (part == 2) {
        const double dres = sqrt(ec[4 * c + 1]);
        k[4] = dres;
        k[7] = dres / (1.0 + s->cnorm);
      } else {
        s->cand_dx2[c] = ec[4 * c + 3];
        s->cand_dy2[c] = er[4 * c + 2];
        s_pre[c] = s->omega * ec[4 * c + 3] + er[4 * c + 2] / s->omega;
        if (c == 0) s_pre[2] = avg ? 1.0 / s->sum_eta : 0.0;
      }
    } else if (part == 3) {
      s_pre[1] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  bool pass[2] = {false, false};
  for (int c = 0; c < 2; ++c) {
    if (c == 1 && !avg) break;
    const double *k = s->kkt[c];
    pass[c] = k[5] <= s->rel_tol && k[6] <= s->rel_tol && k[7] <= s->rel_tol;
  }
  s->inv_avg = s_pre[2];
  if (s->status == kRunning || s->status == kNumErr) {
    if (pass[0]) { s->status = kOptimal; s->ret_which = 0; }
    else if (pass[1]) { s->status = kOptimal; s->ret_which = 1; }
  }
  if (s->status == kRunning) {
    if (s->k >= s->iter_limit) s->status = kIterLimit;
    else if (s->attempts >= s->attempt_limit) s->status = kKktLimit;
    else if (time_up(s)) s->status = kTimeLimit;
  }
  if (s->status == kRunning && s->stall_evals > 0 && s->phase == 1) {
    // the solve has reached what its arithmetic allows when the better
    // candidate's relative error has not dropped by 10% for stall_evals
    // evaluations; it stops and returns that candidate.  (A float32
    // correction problem can keep its relative gap near 1 while its
    // residuals are tiny: its objective terms cancel to below float32
    // resolution; the outer update still gains from such a point.)
    const double e0 = fmax(s->kkt[0][5], fmax(s->kkt[0][6], s->kkt[0][7]));
    const double e1 = avg ? fmax(s->kkt[1][5], fmax(s->kkt[1][6], s->kkt[1][7])) : INFINITY;
    const double err = fmin(e0, e1);
    if (err < 0.9 * s->stall_best) {
      s->stall_best = err;
      s->stall_count = 0;
    } else if (++s->stall_count >= s->stall_evals) {
      s->status = kStalled;
      s->ret_which = e1 < e0 ? 1 : 0;
    }
  }
  s->do_gap = (s->status == kRunning && s->phase == 1 && s->adaptive_restart) ? 1 : 0;
  s->restart = 0;
  s->vrestart = 0;
  if (s->status == kRunning && s->phase == 1 && !s->adaptive_restart && s->pw_update &&
      (double)(s->k - s->k_virt) >= s->beta_art * (double)s->k) {
    // Appendix C.2 "no restart": Algorithm 3 where the artificial criterion
    // would restart, from the point of the previous update (z^{n,0} slots)
    const double Dx = sqrt(s->cand_dx2[0]), Dy = sqrt(s->cand_dy2[0]);
    if (Dx > s->eps_zero && Dy > s->eps_zero)
      s->omega = exp(s->pw_theta * log(Dy / Dx) + (1.0 - s->pw_theta) * log(s->omega));
    s->inv_omega = 1.0 / s->omega;
    s->tau = s->eta * s->inv_omega;
    s->sigma = s->eta * s->omega;
    s->vrestart = 1;
    s->k_virt = s->k;
    double *rec = trace + (size_t)(s->trace_n % kTraceCap) * kTraceLen;
    s->trace_n += 1;
    {
      rec[0] = (double)s->k;
      rec[1] = (double)s->t;
      rec[2] = rec[3] = rec[4] = NAN;
      rec[5] = 0.0;
      rec[6] = 2.0;
      rec[7] = s->omega;
      rec[8] = sqrt(s->omega * s->cand_dx2[0] + s->cand_dy2[0] / s->omega);
      rec[9] = NAN;
      for (int a = 0; a < 3; ++a) {
        rec[10 + a] = s->kkt[0][5 + a];
        rec[13 + a] = s->kkt[1][5 + a];
      }
    }
  }
  if (s->do_gap) {
    // (do_gap needs adaptive restarts: omega did not change above)
    for (int c = 0; c < 2; ++c) {
      const double r2 = s_pre[c];
      s->g_r2[c] = r2;
      s->g_omega[c] = s->omega;
      s->g_inv_omega[c] = s->inv_omega;
      s->g_W[c] = s->g_V[c] = s->g_A[c] = 0.0;
      s->g_prefix[c] = 0u;
      s->g_active[c] = r2 > 0.0 ? 1 : 0;
      s->mu[c] = INFINITY;  // r = 0 gives mu = +inf
      s->gval[c] = 0.0;
    }
  }
  s->phase = 1;
}

}  // namespace pdlp
