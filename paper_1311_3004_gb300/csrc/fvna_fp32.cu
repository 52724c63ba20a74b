// fvna_fp32.cu -- binary32 perturbation-variable kernels (FMA contraction on):
// the packed TMA-fed sweeps of fvna_sweeps32.cuh, their launchers and TMA
// tensor maps, the on-demand budget reduction, and (through
// fvna_precision.inc) the speed pass, drive, import/export and Riemann
// kernels of the binary32 policy.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <new>

#include "fvna_launch.h"
#include "fvna_sweeps32.cuh"
#include "fvna_xh.cuh"

#define POLICY P32
#define SUFFIX fp32
#define HAS_COMP 1
#define FVNA_PRECISION_SWEEPS 0
#include "fvna_precision.inc"

namespace fvna {

// tile_x 16 / 32 / 64 -> halves of 8 / 16 / 32 cells (swizzle span 32 / 64 / 128 B) of the
// tile sweep; tile_x 60 selects the sweep with the lanes along x1 (no tensor maps of its own:
// the maps built for it are those of 32-cell halves, unused)
int x32_half(int tile_x) { return tile_x == 16 ? 8 : tile_x == 32 ? 16 : 32; }

namespace {

typedef void (*StepKernel)(StepArgs);

template <int SW, int LIM> StepKernel px_c(bool comp) {
  return comp ? k_sweep_x32<SW, LIM, true> : k_sweep_x32<SW, LIM, false>;
}
template <int SW> StepKernel px_l(int lim, bool comp) {
  if (lim == LIM_NONE) return px_c<SW, LIM_NONE>(comp);
  if (lim == LIM_LW) return px_c<SW, LIM_LW>(comp);
  return px_c<SW, LIM_MC>(comp);
}
template <int LIM> StepKernel pxh_c(bool comp) {
  return comp ? k_sweep_x32h<LIM, true> : k_sweep_x32h<LIM, false>;
}
StepKernel pxh(int lim, bool comp) {
  if (lim == LIM_NONE) return pxh_c<LIM_NONE>(comp);
  if (lim == LIM_LW) return pxh_c<LIM_LW>(comp);
  return pxh_c<LIM_MC>(comp);
}
// shared memory of the x1 sweep kernel a tile width selects
int smem_x32(int tile_x) { return tile_x == XH_TILE ? 0 : x32_smem_bytes(x32_half(tile_x)); }
StepKernel px(int tile_x, int lim, bool comp) {
  if (tile_x == XH_TILE) return pxh(lim, comp);
  int sw = x32_half(tile_x);
  if (sw == 8) return px_l<8>(lim, comp);
  if (sw == 16) return px_l<16>(lim, comp);
  return px_l<32>(lim, comp);
}
template <int LIM, bool REDO> StepKernel py_c(bool comp) {
  return comp ? k_sweep_y32<LIM, true, REDO> : k_sweep_y32<LIM, false, REDO>;
}
template <bool REDO> StepKernel py(int lim, bool comp) {
  if (lim == LIM_NONE) return py_c<LIM_NONE, REDO>(comp);
  if (lim == LIM_LW) return py_c<LIM_LW, REDO>(comp);
  return py_c<LIM_MC, REDO>(comp);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool make_map(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *m, void *base, const DomDev &d,
              int bx, int by, CUtensorMapSwizzle sw) {
  cuuint64_t dims[2] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny};
  cuuint64_t strides[1] = {(cuuint64_t)d.pitch * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Sum of the stored state of one domain in binary64 (q1 - 1, q2, q3).
__global__ void k_budget32(DomDev D, double *dst) {
  double s[3] = {0.0, 0.0, 0.0};
  const long long n = (long long)D.nx * D.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int j = (int)(c / D.nx), i = (int)(c - (long long)j * D.nx);
    size_t off = (size_t)j * D.pitch + i;
    for (int k = 0; k < 3; k++) s[k] += (double)((const float *)D.qa[k])[off];
  }
  __shared__ double red[3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; k++) {
    double v = warp_sum(s[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < 3; k++) {
      double v = lane < (int)(blockDim.x >> 5) ? red[k][lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) atomicAdd(&dst[k], v);
    }
  }
}

}  // namespace

cudaError_t prepare_kernels_fp32(int tile_x, int lim, int comp) {
  cudaError_t e = cudaFuncSetAttribute(px(tile_x, lim, comp != 0),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_x32(tile_x));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(py<false>(lim, comp != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           y32_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(py<true>(lim, comp != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              y32_smem_bytes());
}

int occupancy_x_fp32(int tile_x, int lim, int comp) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, px(tile_x, lim, comp != 0), 32,
                                                smem_x32(tile_x));
  return n;
}
int occupancy_y_fp32(int lim, int comp) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, py<false>(lim, comp != 0), 32,
                                                y32_smem_bytes());
  return n;
}

// The binary32 sweeps launch as programmatic dependents of the kernel before
// them in the stream (the kernels wait for it before their first global
// access): a sweep's blocks are scheduled while the previous kernel's last
// blocks finish, and in a captured graph the edges between the sweeps are
// programmatic ones.
static cudaError_t launch_dependent(StepKernel k, int blocks, int smem, cudaStream_t s,
                                    const StepArgs &a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a);
}

cudaError_t launch_sweep_x_fp32(int tile_x, const StepArgs &a, int blocks, cudaStream_t s) {
  return launch_dependent(px(tile_x, a.limiter, a.compensated != 0), blocks, smem_x32(tile_x), s,
                          a);
}
cudaError_t launch_sweep_y_fp32(const StepArgs &a, int blocks, cudaStream_t s) {
  return launch_dependent(py<false>(a.limiter, a.compensated != 0), blocks, y32_smem_bytes(), s,
                          a);
}
cudaError_t launch_sweep_y_redo32(const StepArgs &a, int blocks, cudaStream_t s) {
  return launch_dependent(py<true>(a.limiter, a.compensated != 0), blocks, y32_smem_bytes(), s,
                          a);
}

size_t ghost_ring_bytes(int nx, int ny) { return 3 * x2::ghost_ring_size(nx, ny) * sizeof(float); }
cudaError_t launch_ghost32(const StepArgs &a, int dom, int nx, int ny, int always, cudaStream_t s) {
  size_t n = x2::ghost_ring_size(nx, ny);
  int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
  k_ghost32<<<blocks, 256, 0, s>>>(a, dom, always);
  return cudaGetLastError();
}

cudaError_t build_maps_fp32(const DomDev *dd, int n, int tile_x, void **d_maps, cudaStream_t s) {
  *d_maps = nullptr;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const int sw = x32_half(tile_x);
  const CUtensorMapSwizzle swz = sw == 8    ? CU_TENSOR_MAP_SWIZZLE_32B
                                 : sw == 16 ? CU_TENSOR_MAP_SWIZZLE_64B
                                            : CU_TENSOR_MAP_SWIZZLE_128B;
  x2::Maps *h = new (std::nothrow) x2::Maps[n];
  if (!h) return cudaErrorMemoryAllocation;
  bool ok = true;
  for (int d = 0; d < n && ok; d++)
    for (int f = 0; f < 3 && ok; f++) {
      ok = make_map(enc, &h[d].xin[f], dd[d].qa[f], dd[d], sw, X32_ROWS, swz) &&
           make_map(enc, &h[d].xhalo[f], dd[d].qa[f], dd[d], 4, X32_ROWS,
                    CU_TENSOR_MAP_SWIZZLE_NONE) &&
           make_map(enc, &h[d].xout[f], dd[d].qb[f], dd[d], sw, X32_ROWS, swz) &&
           make_map(enc, &h[d].yin[f], dd[d].qb[f], dd[d], x2::YBOX, x2::YRB,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
    }
  if (!ok) {
    delete[] h;
    return cudaErrorInvalidValue;
  }
  void *dm = nullptr;
  cudaError_t e = cudaMalloc(&dm, sizeof(x2::Maps) * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, h, sizeof(x2::Maps) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete[] h;
  if (e != cudaSuccess) {
    cudaFree(dm);
    return e;
  }
  *d_maps = dm;
  return cudaSuccess;
}

cudaError_t launch_budget_fp32(const DomDev &d, double *dst, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dst, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_budget32<<<256, 256, 0, s>>>(d, dst);
  return cudaGetLastError();
}

}  // namespace fvna

#if FVNA_CHECK
extern "C" unsigned long long fvna_check_word() { return fvna::check_word_host(); }
#endif
