// fvna_fp64.cu -- binary64 kernels and the per-step bookkeeping.
//
// Compiled with -fmad=false: no product is fused into a sum, so every
// expression rounds exactly as it is written (the order of the paper's
// definitions, see fvna_device.cuh).  The dt/CFL bookkeeping lives here too,
// because it is binary64 for both precisions (section 4: dt from the CFL
// number of the previous step).
#include "fvna_launch.h"
#include "fvna_step.cuh"
#include "fvna_sweeps.cuh"

#define POLICY P64
#define SUFFIX fp64
#define HAS_COMP 0
#define FVNA_PRECISION_SWEEPS 1
#include "fvna_precision.inc"

namespace fvna {

// End of a step for every domain (see fvna_step.cuh).
__global__ void k_advance(StepArgs A) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < A.ndom) advance_domain(A, d);
}

// Start of a run: time limit and step budget, dt of the first step.
__global__ void k_prepare(StepArgs A, double t_end, long long max_steps) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= A.ndom) return;
  DomScal *S = A.scal + d;
  S->smax_bits = 0ull;
  S->status_bits = 0;
  if (S->status != 0 || max_steps <= 0) {
    S->done = 1;
    return;
  }
  S->done = 0;
  S->timed = t_end > S->t;
  S->t_end = t_end;
  S->steps_left = max_steps;
  if (S->timed && !(S->t < S->t_end)) {
    S->done = 1;
    return;
  }
  S->dt = S->dt_cfl;
  S->last = 0;
  if (S->timed && S->t + S->dt >= S->t_end) {
    S->dt = S->t_end - S->t;
    S->last = 1;
  }
  set_step_scalars(S, A);
}

// After the speed-only pass over the initial state: dt_0 = nu_W dx / max|s|.
__global__ void k_first_dt(StepArgs A) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= A.ndom) return;
  DomScal *S = A.scal + d;
  double s0 = __longlong_as_double((long long)S->smax_bits);
  if (A.dt_fixed <= 0.0 && !(A.doms[d].dt0 > 0.0) && (S->status_bits & ST_NONREAL))
    S->status |= ST_NONREAL;
  const double dt0 = A.doms[d].dt0;
  if (A.dt_fixed > 0.0) S->dt_cfl = A.dt_fixed;
  else if (dt0 > 0.0) S->dt_cfl = dt0;
  else S->dt_cfl = A.nu_w * A.dx / s0;
  S->dt = S->dt_cfl;
  S->smax_bits = 0ull;
  S->status_bits = 0;
  S->nu_min = 1e300;
  set_step_scalars(S, A);
}

// End of a Strang step: the second x1 sweep left the state in the swept
// planes; copy them back (word by word, whatever the precision) for every
// domain still running, and reset the x1 sweep's tile counter (binary32),
// which no x2 sweep resets before the next step.
__global__ void k_copy_back(StepArgs A, int esz) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.counters) A.counters[0] = 0u;
  for (int d = 0; d < A.ndom; d++) {
    if (A.scal[d].done) continue;
    const DomDev &D = A.doms[d];
    const size_t words = (size_t)D.ny * D.pitch * esz / 4;
    for (int k = 0; k < 3; k++) {
      const unsigned *src = (const unsigned *)D.qb[k];
      unsigned *dst = (unsigned *)D.qa[k];
      for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words;
           i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
    }
  }
}

cudaError_t launch_copy_back(const StepArgs &a, int esz, cudaStream_t s) {
  k_copy_back<<<1024, 256, 0, s>>>(a, esz);
  return cudaGetLastError();
}

// Border rule of one side of one domain (fvna_set_bc), in stream order.
__global__ void k_set_bc(DomDev *dd, int dom, int side, int bc) { dd[dom].bc[side] = bc; }

cudaError_t launch_set_bc(DomDev *dd, int dom, int side, int bc, cudaStream_t s) {
  k_set_bc<<<1, 1, 0, s>>>(dd, dom, side, bc);
  return cudaGetLastError();
}
cudaError_t launch_advance(const StepArgs &a, cudaStream_t s) {
  k_advance<<<(a.ndom + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_prepare(const StepArgs &a, double t_end, long long max_steps, cudaStream_t s) {
  k_prepare<<<(a.ndom + 127) / 128, 128, 0, s>>>(a, t_end, max_steps);
  return cudaGetLastError();
}
cudaError_t launch_first_dt(const StepArgs &a, cudaStream_t s) {
  k_first_dt<<<(a.ndom + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fvna
