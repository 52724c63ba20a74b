// fvna_launch3.h -- host-side launchers of the 3D kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "fvna_3d.cuh"

namespace fvna {
namespace d3 {

int tile_x3_64();
int tile_x3_32();
void occupancy3_64(int lim, int comp, int *occ_x, int *occ_v);
void occupancy3_32(int lim, int comp, int *occ_x, int *occ_v);
cudaError_t launch3_sweep_x_64(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_sweep_x_32(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_sweep_v_64(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_sweep_v_32(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_source_64(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_source_32(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_copy_64(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_copy_32(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_speeds_64(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_speeds_32(const Args3 &a, int blocks, cudaStream_t s);
cudaError_t launch3_import_64(const Args3 &a, const double *q, cudaStream_t s);
cudaError_t launch3_import_32(const Args3 &a, const double *q, cudaStream_t s);
cudaError_t launch3_export_64(const Args3 &a, double *q, int what, cudaStream_t s);
cudaError_t launch3_export_32(const Args3 &a, double *q, int what, cudaStream_t s);
cudaError_t launch3_first_dt(const Args3 &a, double dt0, cudaStream_t s);
cudaError_t launch3_prepare(const Args3 &a, double t_end, long long max_steps, cudaStream_t s);
cudaError_t launch3_advance(const Args3 &a, int any_sweep, cudaStream_t s);

}  // namespace d3
}  // namespace fvna
