// fvna_launch.h -- host-side launchers of the step kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "fvna_types.h"

namespace fvna {

constexpr int WARPS_PER_BLOCK = 4;
constexpr int YRING = 8;  // rows in flight per warp in the x2 sweep

// shared memory of one block of each sweep (bytes)
size_t smem_sweep_x(int precision, int tile_x);
size_t smem_sweep_y(int precision);
// one-time attribute setup (opt-in shared memory); returns cudaSuccess or the error
cudaError_t prepare_kernels(int precision, int tile_x, int lim, int comp);
// resident blocks per SM of each sweep
int occupancy_x(int precision, int tile_x, int lim, int comp);
int occupancy_y(int precision, int lim, int comp);

cudaError_t launch_sweep_x(int precision, int tile_x, const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_sweep_y(int precision, const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_advance(const StepArgs &a, cudaStream_t s);
cudaError_t launch_prepare(const StepArgs &a, double t_end, long long max_steps, cudaStream_t s);
cudaError_t launch_speeds(int precision, const StepArgs &a, int dom, cudaStream_t s);
cudaError_t launch_drive(int precision, const StepArgs &a, int dom, int ny, int always,
                         cudaStream_t s);
cudaError_t launch_drive_fp64(const StepArgs &a, int dom, int ny, int always, cudaStream_t s);
cudaError_t launch_drive_fp32(const StepArgs &a, int dom, int ny, int always, cudaStream_t s);
cudaError_t launch_first_dt(const StepArgs &a, cudaStream_t s);
cudaError_t launch_import(int precision, const DomDev &d, const double *q0, cudaStream_t s);
cudaError_t launch_export(int precision, const DomDev &d, double *out, int what, cudaStream_t s);
// end of a Strang step: swept planes back into the state planes (esz: bytes
// per value), the x1 sweep's tile counter reset
cudaError_t launch_copy_back(const StepArgs &a, int esz, cudaStream_t s);
// boundary-flux budget of a sweep (dir 0: x1 sweep, before it; dir 1: x2
// sweep, before it), binary64, added to every domain's outflow; and its reset
cudaError_t launch_border_flux(int precision, const StepArgs &a, int dir, int max_lines,
                               cudaStream_t s);
cudaError_t launch_zero_outflow(const StepArgs &a, cudaStream_t s);
// border rule of one side of one domain in the device descriptors
cudaError_t launch_set_bc(DomDev *dd, int dom, int side, int bc, cudaStream_t s);
// moving domain: shift the window of domain dom by (kx, ky) cells (two
// kernels on s; the device descriptor's corner moves with it)
cudaError_t launch_shift(int precision, const DomDev &d, DomDev *dd, int dom, const DomScal *scal,
                         int kx, int ky, double dx, cudaStream_t s);
cudaError_t launch_shift_fp64(const DomDev &d, DomDev *dd, int dom, const DomScal *scal, int kx,
                              int ky, double dx, cudaStream_t s);
cudaError_t launch_shift_fp32(const DomDev &d, DomDev *dd, int dom, const DomScal *scal, int kx,
                              int ky, double dx, cudaStream_t s);
cudaError_t launch_riemann(int precision, double beta, int n, const double *qL, const double *qR,
                           double *s, double *W, double *am, double *ap, int *nonreal,
                           cudaStream_t st);

// per-precision definitions (fvna_fp64.cu / fvna_fp32.cu)
cudaError_t launch_sweep_x_fp64(int tile_x, const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_sweep_y_fp64(const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_speeds_fp64(const StepArgs &a, int dom, cudaStream_t s);
cudaError_t launch_import_fp64(const DomDev &d, const double *q0, cudaStream_t s);
cudaError_t launch_export_fp64(const DomDev &d, double *out, int what, cudaStream_t s);
cudaError_t launch_riemann_fp64(double beta, int n, const double *qL, const double *qR, double *s,
                                double *W, double *am, double *ap, int *nonreal, cudaStream_t st);
cudaError_t prepare_kernels_fp64(int tile_x, int lim, int comp);
int occupancy_x_fp64(int tile_x, int lim, int comp);
int occupancy_y_fp64(int lim, int comp);

cudaError_t launch_sweep_x_fp32(int tile_x, const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_sweep_y_fp32(const StepArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_speeds_fp32(const StepArgs &a, int dom, cudaStream_t s);
cudaError_t launch_import_fp32(const DomDev &d, const double *q0, cudaStream_t s);
cudaError_t launch_export_fp32(const DomDev &d, double *out, int what, cudaStream_t s);
cudaError_t launch_riemann_fp32(double beta, int n, const double *qL, const double *qR, double *s,
                                double *W, double *am, double *ap, int *nonreal, cudaStream_t st);
cudaError_t prepare_kernels_fp32(int tile_x, int lim, int comp);
int occupancy_x_fp32(int tile_x, int lim, int comp);
int occupancy_y_fp32(int lim, int comp);

// binary32 sweeps (fvna_fp32.cu): x1 tiles are 32 rows x 2*x32_half(tile_x)
// cells, x2 tiles 60 columns x tile_y rows; TMA tensor maps of every domain
// (device array, cudaFree to release); budgets on demand (sum of the state,
// binary64, into dst[3] on the device)
int x32_half(int tile_x);
// tile_x of the binary32 x1 sweep with the lanes along x1 (segments of two rows x 60 cells)
constexpr int X32H_TILE = 60;
constexpr int Y32_COLS = 60;
cudaError_t build_maps_fp32(const DomDev *dd, int n, int tile_x, void **d_maps, cudaStream_t s);
cudaError_t launch_budget_fp32(const DomDev &d, double *dst, cudaStream_t s);
cudaError_t launch_budget_fp64(const DomDev &d, double *dst, cudaStream_t s);
// second kernel of the binary32 x2 sweep (tiles listed for the general split)
cudaError_t launch_sweep_y_redo32(const StepArgs &a, int blocks, cudaStream_t s);
// ghost ring of a binary32 domain with a driven border (bytes), and the
// kernel that fills it with the analytic border values of the current step
size_t ghost_ring_bytes(int nx, int ny);
cudaError_t launch_ghost32(const StepArgs &a, int dom, int nx, int ny, int always, cudaStream_t s);

}  // namespace fvna
