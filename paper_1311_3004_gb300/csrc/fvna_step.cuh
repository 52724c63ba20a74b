// fvna_step.cuh -- the end of a time step for one domain (section 4: the CFL
// number of the step just taken, dt of the next one from max|s|), shared by
// k_advance and by the binary32 x2 sweep's second kernel, which runs it for
// all domains once the sweep is done.  Every binary64 operation is an
// explicitly rounded intrinsic, so the result is the same whatever the
// unit's contraction flags.
#pragma once

#include "fvna_types.h"

namespace fvna {

// Constants of one step derived from dt (dt/dx for the sweeps,
// dt*delta/dx^2 for the source), in binary64 and rounded to binary32 for the
// perturbation kernels.
__device__ __forceinline__ void set_step_scalars(DomScal *S, const StepArgs &A) {
  S->lam = __ddiv_rn(S->dt, A.dx);
  S->coef = __ddiv_rn(__dmul_rn(S->dt, A.delta), __dmul_rn(A.dx, A.dx));
  S->lam32 = (float)S->lam;
  S->coef32 = (float)S->coef;
  S->dt32 = (float)S->dt;
}

// End of a step for domain d: CFL number of the step just taken, the CFL
// statistics (Welford), dt of the next step (nu_W dx / max|s|), time,
// budgets, and whether the run goes on.  A step that would pass t_end is
// shortened to end on it.
__device__ __forceinline__ void advance_domain(const StepArgs &A, int d) {
  DomScal *S = A.scal + d;
  if (S->done) return;
  double smax = __longlong_as_double((long long)S->smax_bits);
  int st = 0;
  if (S->status_bits & ST_NONREAL) st |= ST_NONREAL;
  if (S->status_bits & ST_TIMEOUT) st |= ST_TIMEOUT;
  if (smax != smax) st |= ST_NAN;
  double dt = S->dt;
  if (A.sweeps & 3) {
    double nu = __ddiv_rn(__dmul_rn(dt, smax), A.dx);
    if (nu > A.nu_max) st |= ST_CFL;
    if (!S->last) {
      if (nu < S->nu_min) S->nu_min = nu;
      if (nu > S->nu_max) S->nu_max = nu;
      S->nu_count += 1;
      double dd = __dsub_rn(nu, S->nu_mean);
      S->nu_mean = __dadd_rn(S->nu_mean, __ddiv_rn(dd, (double)S->nu_count));
      S->nu_m2 = __dadd_rn(S->nu_m2, __dmul_rn(dd, __dsub_rn(nu, S->nu_mean)));
    }
  }
  if (A.dt_fixed <= 0.0 && smax > 0.0) S->dt_cfl = __ddiv_rn(__dmul_rn(A.nu_w, A.dx), smax);
  S->dt_last = dt;
  S->smax_last = smax;
  S->t = S->last ? S->t_end : __dadd_rn(S->t, dt);
  S->step += 1;
  for (int k = 0; k < 3; k++) {
    S->budget[k] = S->budget_acc[k];
    S->budget_acc[k] = 0.0;
  }
  S->smax_bits = 0ull;
  S->status_bits = 0;
  S->status |= st;
  if (S->steps_left > 0) S->steps_left -= 1;
  if (S->status != 0 || S->steps_left == 0 || (S->timed && !(S->t < S->t_end))) {
    S->done = 1;
    return;
  }
  S->dt = S->dt_cfl;
  S->last = 0;
  if (S->timed && __dadd_rn(S->t, S->dt) >= S->t_end) {
    S->dt = __dsub_rn(S->t_end, S->t);
    S->last = 1;
  }
  set_step_scalars(S, A);
}

}  // namespace fvna
