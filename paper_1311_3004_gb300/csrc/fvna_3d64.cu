// fvna_3d64.cu -- the 3D step in binary64 total variables (compiled with
// -fmad=false: every expression rounds as written, the order of the
// definitions in fvna_3d.cuh), and the binary64 step bookkeeping of the 3D
// contexts (both precisions).
#include "fvna_3d.cuh"
#include "fvna_launch3.h"

#define T3 double
#define SFX 64
#define HAS_COMP3 0
#include "fvna_3d.inc"

namespace fvna {
namespace d3 {

__global__ void k3_first_dt(Args3 A, double dt0) {
  Scal3 *S = A.S;
  double s0 = __longlong_as_double((long long)S->smax_bits);
  if (A.dt_fixed <= 0.0 && !(dt0 > 0.0) && (S->status_bits & S_NONREAL)) S->status |= S_NONREAL;
  if (A.dt_fixed > 0.0) S->dt_cfl = A.dt_fixed;
  else if (dt0 > 0.0) S->dt_cfl = dt0;
  else S->dt_cfl = __ddiv_rn(__dmul_rn(A.nu_w, A.dx), s0);
  S->dt = S->dt_cfl;
  S->smax_bits = 0ull;
  S->status_bits = 0;
  S->nu_min = 1e300;
  set_scalars3(S, A);
}

__global__ void k3_prepare(Args3 A, double t_end, long long max_steps) {
  Scal3 *S = A.S;
  S->smax_bits = 0ull;
  S->status_bits = 0;
  if (S->status != 0 || max_steps <= 0) { S->done = 1; return; }
  S->done = 0;
  S->timed = t_end > S->t;
  S->t_end = t_end;
  S->steps_left = max_steps;
  if (S->timed && !(S->t < S->t_end)) { S->done = 1; return; }
  S->dt = S->dt_cfl;
  S->last = 0;
  if (S->timed && __dadd_rn(S->t, S->dt) >= S->t_end) {
    S->dt = __dsub_rn(S->t_end, S->t);
    S->last = 1;
  }
  set_scalars3(S, A);
}

// end of a step: CFL number, statistics, dt of the next step, time
__global__ void k3_advance(Args3 A, int any_sweep) {
  Scal3 *S = A.S;
  if (S->done) return;
  double smax = __longlong_as_double((long long)S->smax_bits);
  int st = 0;
  if (S->status_bits & S_NONREAL) st |= S_NONREAL;
  if (smax != smax) st |= S_NAN;
  double dt = S->dt;
  if (any_sweep) {
    double nu = __ddiv_rn(__dmul_rn(dt, smax), A.dx);
    if (nu > A.nu_max) st |= S_CFL;
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
  set_scalars3(S, A);
}

cudaError_t launch3_first_dt(const Args3 &a, double dt0, cudaStream_t s) {
  k3_first_dt<<<1, 1, 0, s>>>(a, dt0);
  return cudaGetLastError();
}
cudaError_t launch3_prepare(const Args3 &a, double t_end, long long max_steps, cudaStream_t s) {
  k3_prepare<<<1, 1, 0, s>>>(a, t_end, max_steps);
  return cudaGetLastError();
}
cudaError_t launch3_advance(const Args3 &a, int any_sweep, cudaStream_t s) {
  k3_advance<<<1, 1, 0, s>>>(a, any_sweep);
  return cudaGetLastError();
}

}  // namespace d3
}  // namespace fvna
