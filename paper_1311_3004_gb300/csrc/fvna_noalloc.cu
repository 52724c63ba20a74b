// fvna_noalloc.cu -- fvna_step_noalloc: one binary64 step that allocates no
// memory.  The paper has no counterpart; this is a deployment convenience.
//
// Some callers cannot allocate device memory on the fly: code that runs with
// a fixed memory budget handed out up front (an embedding application that
// owns every allocation, a process whose allocator is locked down), or a
// real-time loop where a cudaMalloc and its implicit synchronisation are not
// acceptable.  They pass their own input and output planes; everything else
// the step needs (the planes after the x1 sweep, the domain descriptors,
// the per-domain scalars and the warp-tile lists) lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded and
// held by every GPU that loads it until the process exits.
//
// Built with -fmad=false like the other binary64 code: the step is the same
// k_sweep_x / k_sweep_y pair, so its results are identical to fvna_step's.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/fvna.h"
#include "fvna_launch.h"
#include "fvna_sweeps.cuh"

using namespace fvna;

namespace {

constexpr size_t MAX_CELLS = FVNA_NOALLOC_MAX_CELLS;
constexpr int TILE_X = 32;   // x1-sweep tile width used here
constexpr int TILE_Y = 64;   // x2-sweep tile height used here
// Bound on the warp tiles of any nx*ny <= MAX_CELLS domain with nx, ny >= 1:
// ceil(nx/32)*ceil(ny/32) <= MAX_CELLS/1024 + (nx + ny)/32 + 1, and
// ceil(nx/30)*ceil(ny/64) <= MAX_CELLS/1920 + nx/30 + ny/64 + 1.
constexpr size_t MAX_TILES = MAX_CELLS / 1024 + 2 * (MAX_CELLS / 30 + 2) + 2;

// layout of the scratch array (offsets 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_DOM = 0;                                       // DomDev[2]
constexpr size_t OFF_SCAL = align256(OFF_DOM + 2 * sizeof(DomDev)); // DomScal
constexpr size_t OFF_TX = align256(OFF_SCAL + sizeof(DomScal));     // Tile[MAX_TILES]
constexpr size_t OFF_TY = align256(OFF_TX + MAX_TILES * sizeof(Tile));
constexpr size_t OFF_PLANES = align256(OFF_TY + MAX_TILES * sizeof(Tile));
constexpr size_t SCRATCH_BYTES = align256(OFF_PLANES + 3 * MAX_CELLS * sizeof(double));

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once per device with
// that device current (the host-side name g_scratch is only a stand-in).
std::mutex g_mutex;
void *g_addr[256] = {};
int g_blocks_x[256] = {}, g_blocks_y[256] = {};

typedef void (*StepKernel)(StepArgs);
StepKernel kx(int lim) {
  if (lim == LIM_NONE) return k_sweep_x<P64, TILE_X, LIM_NONE, false>;
  if (lim == LIM_LW) return k_sweep_x<P64, TILE_X, LIM_LW, false>;
  return k_sweep_x<P64, TILE_X, LIM_MC, false>;
}
StepKernel ky(int lim) {
  if (lim == LIM_NONE) return k_sweep_y<P64, YRING, LIM_NONE, false>;
  if (lim == LIM_LW) return k_sweep_y<P64, YRING, LIM_LW, false>;
  return k_sweep_y<P64, YRING, LIM_MC, false>;
}

int setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev]) return FVNA_OK;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FVNA_ERR_CUDA;
  size_t smx = (size_t)WARPS_PER_BLOCK * 3 * XROWS * (TILE_X + 2 * HALO_X + 1) * sizeof(double);
  size_t smy = (size_t)WARPS_PER_BLOCK * YRING * 96 * sizeof(double);
  for (int lim = 0; lim < 3; lim++) {
    if (cudaFuncSetAttribute(kx(lim), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx) !=
        cudaSuccess)
      return FVNA_ERR_CUDA;
    if (cudaFuncSetAttribute(ky(lim), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy) !=
        cudaSuccess)
      return FVNA_ERR_CUDA;
  }
  int sms = 0, ox = 0, oy = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FVNA_ERR_CUDA;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ox, kx(LIM_MC), WARPS_PER_BLOCK * 32, smx);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oy, ky(LIM_MC), WARPS_PER_BLOCK * 32, smy);
  g_blocks_x[dev] = (ox > 0 ? ox : 1) * sms;
  g_blocks_y[dev] = (oy > 0 ? oy : 1) * sms;
  g_addr[dev] = p;
  return FVNA_OK;
}

}  // namespace

extern "C" int fvna_step_noalloc(const fvna_config *cfg, const fvna_domain *dom,
                                 const double *q_in, double *q_out, double t, double dt,
                                 double *smax_out, void *stream) {
  if (!cfg || !dom || !q_in || !q_out) return FVNA_ERR_ARG;
  if (cfg->precision != FVNA_FP64) return FVNA_ERR_ARG;
  if (cfg->geometry != FVNA_CARTESIAN && cfg->geometry != FVNA_AXISYMMETRIC) return FVNA_ERR_ARG;
  if (cfg->limiter < FVNA_LIM_MC || cfg->limiter > FVNA_LIM_LW) return FVNA_ERR_ARG;
  if (cfg->sweeps < 0 || cfg->sweeps > 7) return FVNA_ERR_ARG;
  // the same parameter checks as fvna_init, plus a finite time and step
  if (!(cfg->dx > 0.0) || !std::isfinite(cfg->dx)) return FVNA_ERR_ARG;
  if (!std::isfinite(cfg->beta) || !(cfg->delta >= 0.0) || !std::isfinite(cfg->delta))
    return FVNA_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t)) return FVNA_ERR_ARG;
  if (cfg->splitting != FVNA_SPLIT_GODUNOV) return FVNA_ERR_ARG;   // takes the Godunov step
  const int nx = dom->nx, ny = dom->ny;
  if (nx < 1 || ny < 1) return FVNA_ERR_ARG;
  if (dom->bc[0] == FVNA_BC_HIFU && !(dom->focal > 0.0)) return FVNA_ERR_ARG;
  for (int s = 0; s < 4; s++) {
    if (dom->bc[s] < FVNA_BC_PERIODIC || dom->bc[s] > FVNA_BC_HIFU) return FVNA_ERR_ARG;
    int len = s < 2 ? nx : ny;
    if ((dom->bc[s] == FVNA_BC_PERIODIC || dom->bc[s] == FVNA_BC_REFLECT) && len < 3)
      return FVNA_ERR_ARG;
  }
  if ((dom->bc[0] == FVNA_BC_PERIODIC) != (dom->bc[1] == FVNA_BC_PERIODIC)) return FVNA_ERR_ARG;
  if ((dom->bc[2] == FVNA_BC_PERIODIC) != (dom->bc[3] == FVNA_BC_PERIODIC)) return FVNA_ERR_ARG;
  if ((size_t)nx * (size_t)ny > MAX_CELLS) return FVNA_ERR_SIZE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FVNA_ERR_CUDA;
  int rc = setup_device(dev);
  if (rc != FVNA_OK) return rc;
  unsigned char *base = (unsigned char *)g_addr[dev];
  cudaStream_t st = (cudaStream_t)stream;

  // descriptors: the x1 sweep reads q_in and writes the scratch planes, the
  // x2 sweep reads the scratch planes and writes q_out
  DomDev dd[2];
  std::memset(dd, 0, sizeof dd);
  DomDev &g = dd[0];
  g.nx = nx; g.ny = ny; g.pitch = nx; g.env = dom->envelope;
  for (int s = 0; s < 4; s++) g.bc[s] = dom->bc[s];
  g.x0 = dom->x0; g.y0 = dom->y0;
  g.taylor_ratio = dom->taylor_ratio;
  g.taylor_ct = std::cos(dom->taylor_angle);
  g.taylor_st = std::sin(dom->taylor_angle);
  g.amp = dom->amp; g.focal = dom->focal; g.aperture = dom->aperture;
  double *planes = (double *)(base + OFF_PLANES);
  const size_t n = (size_t)nx * ny;
  for (int k = 0; k < 3; k++) {
    g.qa[k] = (void *)(q_in + k * n);
    g.qb[k] = (void *)(planes + k * n);
  }
  dd[1] = g;
  for (int k = 0; k < 3; k++) dd[1].qa[k] = (void *)(q_out + k * n);

  // per-domain scalars: cleared on every call (the array keeps the last
  // call's contents)
  DomScal sc;
  std::memset(&sc, 0, sizeof sc);
  sc.t = t;
  sc.dt = dt;
  sc.dt_cfl = dt;
  sc.done = 0;
  // the same expressions as the device's per-step constants
  sc.lam = dt / cfg->dx;
  sc.coef = dt * cfg->delta / (cfg->dx * cfg->dx);
  sc.lam32 = (float)sc.lam;
  sc.coef32 = (float)sc.coef;
  sc.dt32 = (float)dt;

  // warp tiles (written into the scratch array from this host stack buffer
  // in chunks, so no host allocation either)
  const long long tiles_x = (long long)((nx + TILE_X - 1) / TILE_X) * ((ny + XROWS - 1) / XROWS);
  const long long tiles_y = (long long)((nx + YCOLS - 1) / YCOLS) * ((ny + TILE_Y - 1) / TILE_Y);
  if (tiles_x > (long long)MAX_TILES || tiles_y > (long long)MAX_TILES) return FVNA_ERR_SIZE;
  Tile buf[512];
  int ntx = 0, nty = 0, nb = 0;
  auto flush = [&](size_t off, int first) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(base + off + (size_t)first * sizeof(Tile), buf,
                                    (size_t)nb * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    nb = 0;
    return e;
  };
  cudaError_t e = cudaSuccess;
  int first = 0;
  for (int y = 0; y < ny && e == cudaSuccess; y += XROWS)
    for (int x = 0; x < nx && e == cudaSuccess; x += TILE_X) {
      buf[nb++] = Tile{0, x, y, 0};
      ntx++;
      if (nb == 512) { e = flush(OFF_TX, first); first = ntx; }
    }
  if (e == cudaSuccess && nb) e = flush(OFF_TX, first);
  first = 0;
  for (int y = 0; y < ny && e == cudaSuccess; y += TILE_Y)
    for (int x = 0; x < nx && e == cudaSuccess; x += YCOLS) {
      buf[nb++] = Tile{0, x, y, 0};
      nty++;
      if (nb == 512) { e = flush(OFF_TY, first); first = nty; }
    }
  if (e == cudaSuccess && nb) e = flush(OFF_TY, first);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + OFF_DOM, dd, sizeof dd, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + OFF_SCAL, &sc, sizeof(DomScal), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FVNA_ERR_OOM : FVNA_ERR_CUDA;

  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.doms = (const DomDev *)(base + OFF_DOM);
  a.ndom = 1;
  a.beta = cfg->beta; a.delta = cfg->delta; a.dx = cfg->dx;
  a.nu_w = cfg->nu_w; a.nu_max = cfg->nu_max; a.dt_fixed = dt;
  a.limiter = cfg->limiter; a.geometry = cfg->geometry; a.sweeps = cfg->sweeps;
  a.tile_y = TILE_Y;
  a.scal = (DomScal *)(base + OFF_SCAL);
  // the x1 sweep sees descriptor 0 (q_in -> scratch planes), the x2 sweep
  // descriptor 1 (scratch planes -> q_out); both share the one scalar slot
  StepArgs ax = a, ay = a;
  ax.tiles = (const Tile *)(base + OFF_TX);
  ax.ntiles = ntx;
  ay.doms = (const DomDev *)(base + OFF_DOM) + 1;
  ay.tiles = (const Tile *)(base + OFF_TY);
  ay.ntiles = nty;
  int bx = (ntx + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  int by = (nty + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  bx = bx < g_blocks_x[dev] ? bx : g_blocks_x[dev];
  by = by < g_blocks_y[dev] ? by : g_blocks_y[dev];
  size_t smx = (size_t)WARPS_PER_BLOCK * 3 * XROWS * (TILE_X + 2 * HALO_X + 1) * sizeof(double);
  size_t smy = (size_t)WARPS_PER_BLOCK * YRING * 96 * sizeof(double);
  kx(cfg->limiter)<<<bx, WARPS_PER_BLOCK * 32, smx, st>>>(ax);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    ky(cfg->limiter)<<<by, WARPS_PER_BLOCK * 32, smy, st>>>(ay);
    e = cudaGetLastError();
  }
  DomScal out;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&out, base + OFF_SCAL, sizeof out, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FVNA_ERR_CUDA;
  double smax;
  std::memcpy(&smax, &out.smax_bits, sizeof smax);
  if (smax_out) *smax_out = smax;
  if (out.status_bits & ST_NONREAL) return FVNA_ERR_NONREAL;
  if (smax != smax) return FVNA_ERR_NAN;
  return FVNA_OK;
}
