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

// Boundary-flux budget of one sweep (dir 0: x1 on the state planes, before
// the x1 sweep; dir 1: x2 on the swept planes, before the x2 sweep), in
// binary64 whatever the precision of the state.  Summed over the cells of a
// line, the update of eq. fv-hr telescopes: the fluctuations of two
// neighbouring cells at an inner face add up to f(Q_i) - f(Q_{i-1}) (the Roe
// condition, eq. RoeCond), so the line's sum changes by -dt/dx (Fh_n - Fh_0)
// with the numerical fluxes through its two border faces
//   Fh_0 = f(Q_0) - A+dQ_{-1/2} + F~_{-1/2},   Fh_n = f(Q_{n-1}) + A-dQ_{n-1/2} + F~_{n-1/2}.
// Each thread takes one line and adds dt/dx (Fh_n - Fh_0), in the order
// (q1, q2, q3), to the domain's outflow.  The constant 1 of phi cancels in
// the difference and is left out of f.
template <class P, int LIM>
__global__ void k_border_flux(StepArgs A, int dir) {
  typedef typename P::T T;
  const double beta2 = 2.0 * (A.beta - 1.0);
  for (int d = 0; d < A.ndom; d++) {
    const DomScal *S = A.scal + d;
    if (S->done) continue;
    const DomDev &D = A.doms[d];
    const int n = dir == 0 ? D.nx : D.ny;
    const int lines = dir == 0 ? D.ny : D.nx;
    const double lam = S->lam * (dir == 0 && A.x_half ? 0.5 : 1.0);
    const T *q[3];
    for (int k = 0; k < 3; k++) q[k] = (const T *)(dir == 0 ? D.qa[k] : D.qb[k]);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += gridDim.x * blockDim.x) {
      double fh[2][3];
      for (int side = 0; side < 2; side++) {
        // cells -2..1 (low face between -1 and 0) or n-2..n+1 (high face)
        double c[4][3], zb[4], zc[4];
        for (int m = 0; m < 4; m++) {
          const int g = side == 0 ? m - 2 : n - 2 + m;
          T v[3];
          load_mapped<P>(D, q, dir == 0 ? g : l, dir == 0 ? l : g, S->t, A.dx, v);
          // the sweep's order: (q1, normal momentum, transverse momentum)
          double a = (double)v[0], mn = (double)(dir == 0 ? v[1] : v[2]),
                 mt = (double)(dir == 0 ? v[2] : v[1]);
          c[m][0] = P::pert ? 1.0 + a : a;
          c[m][1] = mn;
          c[m][2] = mt;
          zb[m] = mn / c[m][0];
          zc[m] = mt / c[m][0];
        }
        Iface<double> I[3];
        for (int f = 0; f < 3; f++)
          roe(P64(), beta2, c[f][0], c[f][1], c[f][2], zb[f], zc[f], c[f + 1][0], c[f + 1][1],
              c[f + 1][2], zb[f + 1], zc[f + 1], I[f]);
        FluxData<double> o;
        flux_data<LIM, double>(I[1], I[0], I[2], lam, o);
        // the physical flux of the domain cell next to the face (cell 0 or n-1)
        const double *e = c[side == 0 ? 2 : 1];
        const double a1 = e[0] - 1.0;
        const double f0 = e[1];
        const double f1 = (e[1] / e[0]) * (e[1] / e[0]) + a1 + (A.beta - 1.0) * a1 * a1;
        const double f2 = e[1] * e[2] / (e[0] * e[0]);
        if (side == 0) {
          fh[0][0] = f0 - o.ap[0] + o.F[0];
          fh[0][1] = f1 - o.ap[1] + o.F[1];
          fh[0][2] = f2 - o.ap[2] + o.F[2];
        } else {
          fh[1][0] = f0 + o.am[0] + o.F[0];
          fh[1][1] = f1 + o.am[1] + o.F[1];
          fh[1][2] = f2 + o.am[2] + o.F[2];
        }
      }
      for (int k = 0; k < 3; k++) acc[k] += lam * (fh[1][k] - fh[0][k]);
    }
    // back to (q1, q2, q3): the x2 sweep's normal momentum is q3
    double out[3] = {acc[0], dir == 0 ? acc[1] : acc[2], dir == 0 ? acc[2] : acc[1]};
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 3; k++) {
      double v = warp_sum(out[k]);
      if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
      for (int k = 0; k < 3; k++) {
        double v = lane < (int)(blockDim.x >> 5) ? red[k][lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) atomicAdd(&A.scal[d].outflow[k], v);
      }
    }
    __syncthreads();
  }
}

template <class P> static void launch_bf(const StepArgs &a, int dir, int blocks, cudaStream_t s) {
  if (a.limiter == LIM_NONE) k_border_flux<P, LIM_NONE><<<blocks, 256, 0, s>>>(a, dir);
  else if (a.limiter == LIM_LW) k_border_flux<P, LIM_LW><<<blocks, 256, 0, s>>>(a, dir);
  else k_border_flux<P, LIM_MC><<<blocks, 256, 0, s>>>(a, dir);
}
cudaError_t launch_border_flux(int precision, const StepArgs &a, int dir, int max_lines,
                               cudaStream_t s) {
  int blocks = (max_lines + 255) / 256;
  blocks = blocks < 1 ? 1 : blocks > 64 ? 64 : blocks;
  if (precision == 0) launch_bf<P64>(a, dir, blocks, s);
  else launch_bf<P32>(a, dir, blocks, s);
  return cudaGetLastError();
}

// Sum of the state of one binary64 domain, (q1 - 1, q2, q3), on demand (a
// Strang step ends after the x2 sweep's accumulation of the sum, with the
// second x1 sweep).
__global__ void k_budget64(DomDev D, double *dst) {
  double s[3] = {0.0, 0.0, 0.0};
  const long long n = (long long)D.nx * D.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int j = (int)(c / D.nx), i = (int)(c - (long long)j * D.nx);
    size_t off = (size_t)j * D.pitch + i;
    s[0] += ((const double *)D.qa[0])[off] - 1.0;
    s[1] += ((const double *)D.qa[1])[off];
    s[2] += ((const double *)D.qa[2])[off];
  }
  __shared__ double red[3][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; k++) {
    double v = warp_sum(s[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0)
    for (int k = 0; k < 3; k++) {
      double v = lane < (int)(blockDim.x >> 5) ? red[k][lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) atomicAdd(&dst[k], v);
    }
}
cudaError_t launch_budget_fp64(const DomDev &d, double *dst, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dst, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_budget64<<<256, 256, 0, s>>>(d, dst);
  return cudaGetLastError();
}

// zero the boundary-flux budget of every domain
__global__ void k_zero_outflow(StepArgs A) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < A.ndom)
    for (int k = 0; k < 3; k++) A.scal[d].outflow[k] = 0.0;
}
cudaError_t launch_zero_outflow(const StepArgs &a, cudaStream_t s) {
  k_zero_outflow<<<(a.ndom + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
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
