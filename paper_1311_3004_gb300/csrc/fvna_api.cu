// fvna_api.cu -- host runtime behind include/fvna.h.
//
// A context owns, per domain, two sets of three SoA planes (the state and the
// planes after the x1 sweep), rows padded to 32 elements; one array of
// domain descriptors and one of per-domain device scalars (time, dt, CFL
// statistics, status, budgets); and the two warp-tile lists of the sweeps.
// A step is three launches on the caller's stream: the x1 sweep, the fused
// x2 sweep + source, and the per-domain dt update.  Steps are captured once
// into a CUDA graph of `steps_per_graph` steps and replayed; the kernels of a
// finished domain return at once, so a replay may overrun the end of a run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fvna.h"
#include "fvna_launch.h"
#include "fvna_net.h"

using namespace fvna;

struct fvna_ctx {
  fvna_config cfg;
  int ndom = 0;
  std::vector<fvna_domain> doms;
  std::vector<DomDev> dd;
  DomDev *d_dd = nullptr;
  DomScal *d_scal = nullptr;
  Tile *d_tx = nullptr, *d_ty = nullptr;
  int ntx = 0, nty = 0;
  void *d_state = nullptr;
  double *d_stage = nullptr;  // staging for host<->device state copies
  size_t stage_bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 32;
  int tile_x = 32, tile_y = 64;
  int blocks_x = 1, blocks_y = 1;
  StepArgs args;    // common arguments (no tile list)
  StepArgs args_x;  // x1 sweep: warp tiles of 32 rows x tile_x cells
  StepArgs args_y;  // x2 sweep: warp tiles of 30 columns x tile_y rows
  DomScal *h_scal = nullptr;  // pinned mirror
  long long launches = 0;
  int kernels_per_step = 3;
  // learned correction applied after every step (single FP32 domain)
  fvna_net *net = nullptr;
  float net_in = 1.f, net_out = 1.f;
  int net_every = 1;
  int net_band = 0;
  __nv_bfloat16 *net_h = nullptr;   // two hidden activation buffers
  void *d_maps = nullptr;           // binary32: TMA tensor maps of every domain
  unsigned *d_ctr = nullptr;        // binary32: tile counters of the two sweeps
  int *d_redo = nullptr;            // binary32: x2-sweep tiles listed for the general split
  int redo_blocks = 1;
  double *d_budget = nullptr;       // on-demand budget sums (binary32, binary64 Strang)
  // moving domain: whole cells each window has moved since init (x1, x2)
  std::vector<long long> moved_x, moved_y;
  // boundary-flux budgets (fvna_set_budgets): one small kernel before each sweep
  int budgets = 0;
  int max_lines = 1;
};

namespace {

cudaError_t g_last_cuda_error = cudaSuccess;

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return FVNA_OK;
  g_last_cuda_error = e;
  if (e == cudaErrorMemoryAllocation) return FVNA_ERR_OOM;
  return FVNA_ERR_CUDA;
}

#define CK(call)                                \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_err(e_); \
  } while (0)

int status_code(int bits) {
  if (bits & ST_TIMEOUT) return FVNA_ERR_TIMEOUT;
  if (bits & ST_NONREAL) return FVNA_ERR_NONREAL;
  if (bits & ST_NAN) return FVNA_ERR_NAN;
  if (bits & ST_CFL) return FVNA_ERR_CFL;
  return FVNA_OK;
}

bool valid_bc(int b) { return b >= BC_PERIODIC && b <= BC_HIFU; }

int validate(const fvna_config *c, int n, const fvna_domain *d, const double *const *q0) {
  if (!c || n < 1 || !d || !q0) return FVNA_ERR_ARG;
  if (c->precision != FVNA_FP64 && c->precision != FVNA_FP32_PERT) return FVNA_ERR_ARG;
  if (c->geometry != FVNA_CARTESIAN && c->geometry != FVNA_AXISYMMETRIC) return FVNA_ERR_ARG;
  if (c->limiter < FVNA_LIM_MC || c->limiter > FVNA_LIM_LW) return FVNA_ERR_ARG;
  if (c->sweeps < 0 || c->sweeps > 7) return FVNA_ERR_ARG;
  if (!(c->dx > 0.0) || !std::isfinite(c->dx)) return FVNA_ERR_ARG;
  if (!std::isfinite(c->beta) || !(c->delta >= 0.0) || !std::isfinite(c->delta)) return FVNA_ERR_ARG;
  if (!(c->dt_fixed > 0.0) && !(c->nu_w > 0.0)) return FVNA_ERR_ARG;
  if (!(c->nu_max > 0.0)) return FVNA_ERR_ARG;
  if (c->steps_per_graph < 0 || c->steps_per_graph > 4096) return FVNA_ERR_ARG;
  if (c->tile_x != 0 && c->tile_x != 16 && c->tile_x != 32 && c->tile_x != 64 &&
      !(c->tile_x == X32H_TILE && c->precision == FVNA_FP32_PERT))
    return FVNA_ERR_ARG;
  if (c->tile_y != 0 && (c->tile_y < 8 || c->tile_y > 4096)) return FVNA_ERR_ARG;
  if (c->compensated != 0 && c->compensated != 1) return FVNA_ERR_ARG;
  if (c->splitting != FVNA_SPLIT_GODUNOV && c->splitting != FVNA_SPLIT_STRANG) return FVNA_ERR_ARG;
  for (int k = 0; k < n; k++) {
    const fvna_domain &D = d[k];
    if (D.nx < 1 || D.ny < 1 || D.nx > (1 << 20) || D.ny > (1 << 20)) return FVNA_ERR_ARG;
    if ((long long)D.nx * D.ny > (1ll << 33)) return FVNA_ERR_ARG;
    if (!q0[k]) return FVNA_ERR_ARG;
    for (int s = 0; s < 4; s++) {
      if (!valid_bc(D.bc[s])) return FVNA_ERR_ARG;
      int len = s < 2 ? D.nx : D.ny;
      if ((D.bc[s] == BC_PERIODIC || D.bc[s] == BC_REFLECT) && len < 3) return FVNA_ERR_ARG;
    }
    // periodic borders come in pairs
    if ((D.bc[0] == BC_PERIODIC) != (D.bc[1] == BC_PERIODIC)) return FVNA_ERR_ARG;
    if ((D.bc[2] == BC_PERIODIC) != (D.bc[3] == BC_PERIODIC)) return FVNA_ERR_ARG;
    if (D.bc[0] == BC_HIFU && !(D.focal > 0.0)) return FVNA_ERR_ARG;
    if (!(D.dt0 >= 0.0) || !std::isfinite(D.t0)) return FVNA_ERR_ARG;
  }
  return FVNA_OK;
}

void free_ctx(fvna_ctx *c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaFree(c->d_dd);
  cudaFree(c->d_scal);
  cudaFree(c->d_tx);
  cudaFree(c->d_ty);
  cudaFree(c->d_state);
  cudaFree(c->d_stage);
  cudaFree(c->net_h);
  cudaFree(c->d_maps);
  cudaFree(c->d_ctr);
  cudaFree(c->d_redo);
  cudaFree(c->d_budget);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
}

// border values of the step: the HIFU drive buffer (binary64 domains) or
// the ghost ring (binary32 domains with a driven border)
int enqueue_drives(fvna_ctx *c, cudaStream_t s) {
  for (int d = 0; d < c->ndom; d++) {
    if (c->dd[d].drive) CK(launch_drive(c->cfg.precision, c->args, d, c->dd[d].ny, 0, s));
    if (c->dd[d].ghost32) CK(launch_ghost32(c->args, d, c->dd[d].nx, c->dd[d].ny, 0, s));
  }
  return FVNA_OK;
}

// a sweep: binary64 one kernel; binary32 x1 one kernel (a tile that meets a
// face that is not subsonic is redone inside it), binary32 x2 the
// speculative kernel, then the kernel that redoes the tiles it listed
// (usually none: it returns at once)
cudaError_t sweep_x(fvna_ctx *c, cudaStream_t s) {
  if (c->budgets) {
    cudaError_t e = launch_border_flux(c->cfg.precision, c->args_x, 0, c->max_lines, s);
    if (e != cudaSuccess) return e;
  }
  return launch_sweep_x(c->cfg.precision, c->tile_x, c->args_x, c->blocks_x, s);
}
cudaError_t sweep_y(fvna_ctx *c, cudaStream_t s) {
  if (c->budgets) {
    cudaError_t e = launch_border_flux(c->cfg.precision, c->args_y, 1, c->max_lines, s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_sweep_y(c->cfg.precision, c->args_y, c->blocks_y, s);
  if (e == cudaSuccess && c->cfg.precision == FVNA_FP32_PERT)
    e = launch_sweep_y_redo32(c->args_y, c->redo_blocks, s);
  return e;
}

int enqueue_steps_raw(fvna_ctx *c, cudaStream_t s, int nsteps) {
  for (int i = 0; i < nsteps; i++) {
    int rc = enqueue_drives(c, s);
    if (rc != FVNA_OK) return rc;
    CK(sweep_x(c, s));
    CK(sweep_y(c, s));
    if (c->cfg.splitting == FVNA_SPLIT_STRANG) {
      // the second half x1 sweep, then its result back into the state planes
      CK(sweep_x(c, s));
      CK(launch_copy_back(c->args, c->cfg.precision == FVNA_FP64 ? 8 : 4, s));
    }
    if (c->net) {
      const DomDev &d = c->dd[0];
      size_t pix = (size_t)d.nx * d.ny;
      long long pstride = (long long)(((char *)d.qa[1] - (char *)d.qa[0]) / sizeof(float));
      CK(net_forward_launch(c->net, 1, d.ny, d.nx, (const float *)d.qa[0], pstride, d.pitch, 0,
                            c->net_in, (float *)d.qa[0], pstride, d.pitch, 0, 1, c->net_out,
                            c->net_h, c->net_h + pix * 32, s, &c->d_scal[0].done,
                            &c->d_scal[0].step, c->net_every, c->net_band));
    }
    if (!c->args_y.fold_advance) CK(launch_advance(c->args, s));
  }
  return FVNA_OK;
}

int ensure_graph(fvna_ctx *c) {
  if (c->gexec) return FVNA_OK;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_steps_raw(c, c->cap, c->gsteps);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (rc != FVNA_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(e);
  c->graph = g;
  CK(cudaGraphInstantiate(&c->gexec, g, 0));
  return FVNA_OK;
}

int launch_graphs(fvna_ctx *c, long long n) {
  for (long long i = 0; i < n; i++) {
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->launches += (long long)c->gsteps * c->kernels_per_step;
  }
  return FVNA_OK;
}

int read_scal(fvna_ctx *c) {
  CK(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(DomScal) * c->ndom, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return FVNA_OK;
}

int first_status(const fvna_ctx *c) {
  for (int d = 0; d < c->ndom; d++) {
    int s = status_code(c->h_scal[d].status);
    if (s != FVNA_OK) return s;
  }
  return FVNA_OK;
}

void fill_stats(const DomScal &S, fvna_stats *st) {
  st->steps = S.step;
  st->t = S.t;
  st->dt = S.dt_cfl;
  st->dt_last = S.dt_last;
  st->smax = S.smax_last;
  double n = S.nu_count > 0 ? (double)S.nu_count : 1.0;
  st->nu_min = S.nu_count > 0 ? S.nu_min : 0.0;
  st->nu_max = S.nu_count > 0 ? S.nu_max : 0.0;
  st->nu_mean = S.nu_mean;
  double var = S.nu_m2 / n;
  st->nu_std = var > 0.0 ? std::sqrt(var) : 0.0;
  st->status = status_code(S.status);
  st->reserved = 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// launch dispatch by precision
// ---------------------------------------------------------------------------
namespace fvna {
cudaError_t prepare_kernels(int p, int tx, int lim, int comp) {
  return p == FVNA_FP64 ? prepare_kernels_fp64(tx, lim, comp) : prepare_kernels_fp32(tx, lim, comp);
}
int occupancy_x(int p, int tx, int lim, int comp) {
  return p == FVNA_FP64 ? occupancy_x_fp64(tx, lim, comp) : occupancy_x_fp32(tx, lim, comp);
}
int occupancy_y(int p, int lim, int comp) {
  return p == FVNA_FP64 ? occupancy_y_fp64(lim, comp) : occupancy_y_fp32(lim, comp);
}
cudaError_t launch_sweep_x(int p, int tx, const StepArgs &a, int b, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_sweep_x_fp64(tx, a, b, s) : launch_sweep_x_fp32(tx, a, b, s);
}
cudaError_t launch_sweep_y(int p, const StepArgs &a, int b, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_sweep_y_fp64(a, b, s) : launch_sweep_y_fp32(a, b, s);
}
cudaError_t launch_speeds(int p, const StepArgs &a, int dom, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_speeds_fp64(a, dom, s) : launch_speeds_fp32(a, dom, s);
}
cudaError_t launch_drive(int p, const StepArgs &a, int dom, int ny, int always, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_drive_fp64(a, dom, ny, always, s)
                        : launch_drive_fp32(a, dom, ny, always, s);
}
cudaError_t launch_import(int p, const DomDev &d, const double *q0, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_import_fp64(d, q0, s) : launch_import_fp32(d, q0, s);
}
cudaError_t launch_export(int p, const DomDev &d, double *out, int what, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_export_fp64(d, out, what, s) : launch_export_fp32(d, out, what, s);
}
cudaError_t launch_shift(int p, const DomDev &d, DomDev *dd, int dom, const DomScal *scal, int kx,
                         int ky, double dx, cudaStream_t s) {
  return p == FVNA_FP64 ? launch_shift_fp64(d, dd, dom, scal, kx, ky, dx, s)
                        : launch_shift_fp32(d, dd, dom, scal, kx, ky, dx, s);
}
cudaError_t launch_riemann(int p, double beta, int n, const double *qL, const double *qR, double *s,
                           double *W, double *am, double *ap, int *nr, cudaStream_t st) {
  return p == FVNA_FP64 ? launch_riemann_fp64(beta, n, qL, qR, s, W, am, ap, nr, st)
                        : launch_riemann_fp32(beta, n, qL, qR, s, W, am, ap, nr, st);
}
}  // namespace fvna

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *fvna_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda_error); }

const char *fvna_strerror(int code) {
  switch (code) {
    case FVNA_OK: return "ok";
    case FVNA_ERR_ARG: return "invalid argument";
    case FVNA_ERR_CUDA: return "CUDA runtime error";
    case FVNA_ERR_OOM: return "device out of memory";
    case FVNA_ERR_NONREAL: return "non-real wave speeds (state outside the hyperbolic region)";
    case FVNA_ERR_CFL: return "CFL number above nu_max";
    case FVNA_ERR_NAN: return "NaN wave speed";
    case FVNA_ERR_SIZE: return "domain larger than the fixed scratch area allows";
    case FVNA_ERR_TIMEOUT: return "a kernel timed out waiting for its own asynchronous copy";
    default: return "unknown status";
  }
}

// Tile shapes of the binary32 sweeps when the configuration leaves them
// open.  Each SM works through ceil(tiles / SMs) tiles whose cost grows with
// the cells a lane marches (tile plus halo); fewer than `want` tiles per SM
// leave the SM short of warps to overlap, which the cost counts as idle.
static double tile_cost(long long tiles, int sms, int per_tile, int want) {
  double per_sm = std::ceil((double)tiles / sms);
  double fill = std::min(1.0, (double)tiles / sms / want);
  return per_sm * per_tile / fill;
}
static int pick_tile_x32(int n, const fvna_domain *d, int sms) {
  int best = 64;
  double best_cost = 1e300;
  for (int tx : {64, 32, 16}) {
    int sw = x32_half(tx);
    long long T = 0;
    for (int k = 0; k < n; k++)
      T += (long long)((d[k].ny + XROWS - 1) / XROWS) * ((d[k].nx + 2 * sw - 1) / (2 * sw));
    double c = tile_cost(T, sms, sw + 4, 7);
    if (c < best_cost) { best_cost = c; best = tx; }
  }
  return best;
}
// x2 sweep: each warp marches its columns row after row, so the sweep runs
// at the pace of its warps' latency and of its slowest tiles (those at a
// border take the general path); a height whose marched rows (ty + 6) fill
// whole 8-row chunks.  The smallest, 10 (two chunks, both loaded when the
// tile starts, and the most tiles to balance the warps with), measured
// fastest on the 2048^2 pulse (53.6 us against 56.2 for 18 and 68.7 for 22;
// taller tiles and mixed heights were slower still).
static int pick_tile_y32() { return 10; }

static int init_impl(const fvna_config *cfg, int n, const fvna_domain *doms,
                     const double *const *q0, int q0_on_device, void *stream, fvna_ctx *c) {
  c->cfg = *cfg;
  c->ndom = n;
  c->doms.assign(doms, doms + n);
  c->stream = (cudaStream_t)stream;
  const int prec = cfg->precision;
  const size_t esz = prec == FVNA_FP64 ? sizeof(double) : sizeof(float);
  c->gsteps = cfg->steps_per_graph > 0 ? cfg->steps_per_graph : 32;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (prec == FVNA_FP64) {
    c->tile_x = cfg->tile_x ? cfg->tile_x : 32;
    c->tile_y = cfg->tile_y ? cfg->tile_y : 64;
  } else {
    c->tile_x = cfg->tile_x ? cfg->tile_x : pick_tile_x32(n, doms, sms);
    c->tile_y = cfg->tile_y ? cfg->tile_y : pick_tile_y32();
  }
  // border values evaluated once per step: binary64 domains driven on the
  // x1-low border (HIFU) keep a drive buffer; binary32 domains with any
  // driven border (Taylor, HIFU) a ghost ring
  auto driven = [&](const fvna_domain &D) {
    for (int k = 0; k < 4; k++)
      if (D.bc[k] == BC_TAYLOR) return true;
    return D.bc[0] == BC_HIFU;
  };
  auto border_bytes = [&](const fvna_domain &D) -> size_t {
    if (prec == FVNA_FP64)
      return D.bc[0] == BC_HIFU ? (3 * HALO_Y * (size_t)D.ny * esz + 255) / 256 * 256 : 0;
    return driven(D) ? (ghost_ring_bytes(D.nx, D.ny) + 255) / 256 * 256 : 0;
  };
  c->kernels_per_step = 3;
  for (int d = 0; d < n; d++) c->kernels_per_step += border_bytes(doms[d]) ? 1 : 0;

  // state planes: 2 sets x 3 planes per domain, each plane 256-byte aligned,
  // then the domain's border buffer
  std::vector<size_t> offs(n), doffs(n);
  size_t total = 0, max_cells = 0;
  for (int d = 0; d < n; d++) {
    size_t pitch = ((size_t)doms[d].nx + 31) / 32 * 32;
    size_t plane = (pitch * doms[d].ny * esz + 255) / 256 * 256;
    offs[d] = total;
    total += 6 * plane;
    doffs[d] = total;
    total += border_bytes(doms[d]);
    max_cells = std::max(max_cells, (size_t)doms[d].nx * doms[d].ny);
  }
  CK(cudaMalloc(&c->d_state, total));
  CK(cudaMalloc(&c->d_budget, 3 * sizeof(double)));
  for (int d = 0; d < n; d++) c->max_lines = std::max(c->max_lines, std::max(doms[d].nx, doms[d].ny));
  c->dd.resize(n);
  c->moved_x.assign(n, 0);
  c->moved_y.assign(n, 0);
  for (int d = 0; d < n; d++) {
    const fvna_domain &D = doms[d];
    DomDev &g = c->dd[d];
    std::memset(&g, 0, sizeof g);
    g.nx = D.nx; g.ny = D.ny;
    g.pitch = (D.nx + 31) / 32 * 32;
    g.env = D.envelope;
    for (int s = 0; s < 4; s++) g.bc[s] = D.bc[s];
    g.x0 = D.x0; g.y0 = D.y0;
    g.taylor_ratio = D.taylor_ratio;
    g.taylor_ct = std::cos(D.taylor_angle);
    g.taylor_st = std::sin(D.taylor_angle);
    g.amp = D.amp; g.focal = D.focal; g.aperture = D.aperture;
    g.dt0 = D.dt0;
    size_t plane = ((size_t)g.pitch * D.ny * esz + 255) / 256 * 256;
    char *base = (char *)c->d_state + offs[d];
    for (int k = 0; k < 3; k++) {
      g.qa[k] = base + k * plane;
      g.qb[k] = base + (3 + k) * plane;
    }
    char *bb = border_bytes(D) ? (char *)c->d_state + doffs[d] : nullptr;
    g.drive = prec == FVNA_FP64 ? bb : nullptr;
    g.ghost32 = prec == FVNA_FP64 ? nullptr : bb;
  }
  CK(cudaMemsetAsync(c->d_state, 0, total, c->stream));
  CK(cudaMalloc(&c->d_dd, sizeof(DomDev) * n));
  CK(cudaMemcpyAsync(c->d_dd, c->dd.data(), sizeof(DomDev) * n, cudaMemcpyHostToDevice, c->stream));
  std::vector<DomScal> sc(n);
  for (int d = 0; d < n; d++) {
    std::memset(&sc[d], 0, sizeof(DomScal));
    sc[d].t = doms[d].t0;
    sc[d].nu_min = 1e300;
    sc[d].done = 1;
  }
  CK(cudaMalloc(&c->d_scal, sizeof(DomScal) * n));
  CK(cudaMemcpyAsync(c->d_scal, sc.data(), sizeof(DomScal) * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMallocHost(&c->h_scal, sizeof(DomScal) * n));

  // warp tiles (binary64: 32 rows x tile_x and 30 columns x tile_y;
  // binary32: 32 rows x 2 halves and 60 columns x tile_y)
  // (binary32: the tiles that touch a domain border come first; they take
  // longer and the sweeps hand tiles out in list order)
  std::vector<Tile> tx, ty, txb, tyb;
  const int sw = x32_half(c->tile_x);
  // binary32 x1 sweep with the lanes along x1: segments of two rows x 60 cells
  const bool xh = prec == FVNA_FP32_PERT && c->tile_x == X32H_TILE;
  const int xstep = prec == FVNA_FP64 ? c->tile_x : xh ? X32H_TILE : 2 * sw;
  const int xrows = xh ? 2 : XROWS;
  const int ystep = prec == FVNA_FP64 ? YCOLS : Y32_COLS;
  for (int d = 0; d < n; d++) {
    const int nx = doms[d].nx, ny = doms[d].ny;
    for (int y = 0; y < ny; y += xrows)
      for (int x = 0; x < nx; x += xstep) {
        bool b = xh ? (x < 2 || x + X32H_TILE + 2 > nx || y + 2 > ny)
                    : prec == FVNA_FP32_PERT && (x == 0 || x + 2 * sw + 2 > nx || y + XROWS > ny);
        (b ? txb : tx).push_back(Tile{d, x, y, 0});
      }
    for (int y = 0; y < ny; y += c->tile_y)
      for (int x = 0; x < nx; x += ystep) {
        bool b = prec == FVNA_FP32_PERT &&
                 (x < 2 || x + Y32_COLS + 2 > nx || y < HALO_Y || y + c->tile_y + HALO_Y > ny);
        (b ? tyb : ty).push_back(Tile{d, x, y, 0});
      }
  }
  tx.insert(tx.begin(), txb.begin(), txb.end());
  ty.insert(ty.begin(), tyb.begin(), tyb.end());
  c->ntx = (int)tx.size();
  c->nty = (int)ty.size();
  CK(cudaMalloc(&c->d_tx, sizeof(Tile) * tx.size()));
  CK(cudaMalloc(&c->d_ty, sizeof(Tile) * ty.size()));
  CK(cudaMemcpyAsync(c->d_tx, tx.data(), sizeof(Tile) * tx.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_ty, ty.data(), sizeof(Tile) * ty.size(), cudaMemcpyHostToDevice, c->stream));

  // kernel set-up and persistent grid sizes
  const int comp = prec == FVNA_FP32_PERT && cfg->compensated ? 1 : 0;
  CK(prepare_kernels(prec, c->tile_x, cfg->limiter, comp));
  int occx = std::max(1, occupancy_x(prec, c->tile_x, cfg->limiter, comp));
  int occy = std::max(1, occupancy_y(prec, cfg->limiter, comp));
  const int wpb = prec == FVNA_FP64 ? WARPS_PER_BLOCK : 1;  // binary32: one warp per block
  c->blocks_x = std::max(1, std::min((c->ntx + wpb - 1) / wpb, occx * sms));
  c->blocks_y = std::max(1, std::min((c->nty + wpb - 1) / wpb, occy * sms));
  if (prec == FVNA_FP32_PERT) {
    CK(build_maps_fp32(c->dd.data(), n, c->tile_x, &c->d_maps, c->stream));
    CK(cudaMalloc(&c->d_ctr, 3 * sizeof(unsigned)));
    CK(cudaMemsetAsync(c->d_ctr, 0, 3 * sizeof(unsigned), c->stream));
    CK(cudaMalloc(&c->d_redo, (2 + (size_t)c->nty) * sizeof(int)));
    CK(cudaMemsetAsync(c->d_redo, 0, 2 * sizeof(int), c->stream));
    c->redo_blocks = sms;
    // x1 sweep, x2 sweep and its second kernel, which ends the step
  }

  StepArgs &a = c->args;
  std::memset(&a, 0, sizeof a);
  a.doms = c->d_dd;
  a.scal = c->d_scal;
  a.ndom = n;
  a.beta = cfg->beta; a.delta = cfg->delta; a.dx = cfg->dx;
  a.nu_w = cfg->nu_w; a.nu_max = cfg->nu_max; a.dt_fixed = cfg->dt_fixed;
  a.limiter = cfg->limiter; a.geometry = cfg->geometry; a.sweeps = cfg->sweeps;
  a.tile_y = c->tile_y;
  a.compensated = comp;
  a.wait_polls = cfg->wait_limit == 0 ? (1 << 22) : cfg->wait_limit < 0 ? 0 : cfg->wait_limit;
  a.tmaps = c->d_maps;
  a.counters = c->d_ctr;
  a.redo = c->d_redo;
  c->args_x = a;
  c->args_x.tiles = c->d_tx;
  c->args_x.ntiles = c->ntx;
  c->args_x.sweep = 0;
  c->args_y = a;
  c->args_y.tiles = c->d_ty;
  c->args_y.ntiles = c->nty;
  c->args_y.redo_off = 2;
  c->args_y.sweep = 1;
  // Strang: the step ends after the second x1 sweep, so never in the x2 sweep
  const bool strang = cfg->splitting == FVNA_SPLIT_STRANG;
  c->args_x.x_half = strang ? 1 : 0;
  c->args_y.fold_advance = prec == FVNA_FP32_PERT && !strang ? 1 : 0;
  if (strang) c->kernels_per_step += prec == FVNA_FP32_PERT ? 3 : 2;


  // initial state
  if (!q0_on_device) {
    c->stage_bytes = max_cells * 3 * sizeof(double);
    CK(cudaMalloc(&c->d_stage, c->stage_bytes));
  }
  for (int d = 0; d < n; d++) {
    const double *src = q0[d];
    size_t bytes = (size_t)doms[d].nx * doms[d].ny * 3 * sizeof(double);
    if (!q0_on_device) {
      CK(cudaMemcpyAsync(c->d_stage, q0[d], bytes, cudaMemcpyHostToDevice, c->stream));
      src = c->d_stage;
    }
    CK(launch_import(prec, c->dd[d], src, c->stream));
  }
  // the speed pass reads the border values of the initial time
  for (int d = 0; d < n; d++) {
    if (c->dd[d].drive) CK(launch_drive(prec, a, d, doms[d].ny, 1, c->stream));
    // speeds of the initial state -> first dt
    StepArgs sa = a;
    CK(launch_speeds(prec, sa, d, c->stream));
  }
  CK(launch_first_dt(a, c->stream));
  CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(c->stream));
  return FVNA_OK;
}

int fvna_init(const fvna_config *cfg, int n_domains, const fvna_domain *doms,
              const double *const *q0, int q0_on_device, void *stream, fvna_ctx **out) {
  if (!out) return FVNA_ERR_ARG;
  *out = nullptr;
  int v = validate(cfg, n_domains, doms, q0);
  if (v != FVNA_OK) return v;
  fvna_ctx *c = new (std::nothrow) fvna_ctx();
  if (!c) return FVNA_ERR_OOM;
  int rc = init_impl(cfg, n_domains, doms, q0, q0_on_device, stream, c);
  if (rc != FVNA_OK) {
    cudaGetLastError();
    free_ctx(c);
    return rc;
  }
  *out = c;
  return FVNA_OK;
}

int fvna_step(fvna_ctx *c, long long nsteps) {
  if (!c || nsteps < 0) return FVNA_ERR_ARG;
  if (nsteps == 0) return FVNA_OK;
  int rc = ensure_graph(c);
  if (rc != FVNA_OK) return rc;
  CK(launch_prepare(c->args, -1e300, nsteps, c->stream));
  c->launches += 1;
  return launch_graphs(c, (nsteps + c->gsteps - 1) / c->gsteps);
}

int fvna_run(fvna_ctx *c, double t_end, long long max_steps, fvna_stats *stats) {
  if (!c || max_steps < 0) return FVNA_ERR_ARG;
  int rc = ensure_graph(c);
  if (rc != FVNA_OK) return rc;
  CK(launch_prepare(c->args, t_end, max_steps, c->stream));
  c->launches += 1;
  long long left = max_steps > 0 ? (max_steps + c->gsteps - 1) / c->gsteps : 0;
  long long batch = 1;
  while (left > 0) {
    long long nb = std::min(batch, left);
    rc = launch_graphs(c, nb);
    if (rc != FVNA_OK) return rc;
    left -= nb;
    rc = read_scal(c);
    if (rc != FVNA_OK) return rc;
    bool all_done = true;
    for (int d = 0; d < c->ndom; d++) all_done &= c->h_scal[d].done != 0;
    if (all_done) break;
    batch = std::min<long long>(batch * 2, 64);
  }
  rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  if (stats) fill_stats(c->h_scal[0], stats);
  return first_status(c);
}

int fvna_shift(fvna_ctx *c, int domain, int kx, int ky) {
  if (!c || domain < 0 || domain >= c->ndom) return FVNA_ERR_ARG;
  const fvna_domain &D = c->doms[domain];
  if (kx <= -D.nx || kx >= D.nx || ky <= -D.ny || ky >= D.ny) return FVNA_ERR_ARG;
  if (ky != 0 && c->cfg.geometry == FVNA_AXISYMMETRIC) return FVNA_ERR_ARG;
  if (kx == 0 && ky == 0) return FVNA_OK;
  CK(launch_shift(c->cfg.precision, c->dd[domain], c->d_dd, domain, c->d_scal, kx, ky, c->cfg.dx,
                  c->stream));
  c->launches += 2;
  c->moved_x[domain] += kx;
  c->moved_y[domain] += ky;
  return FVNA_OK;
}

int fvna_set_bc(fvna_ctx *c, int domain, int side, int bc) {
  if (!c || domain < 0 || domain >= c->ndom || side < 0 || side > 3 || !valid_bc(bc))
    return FVNA_ERR_ARG;
  fvna_domain D = c->doms[domain];
  D.bc[side] = bc;
  const int len = side < 2 ? D.nx : D.ny;
  if ((bc == BC_PERIODIC || bc == BC_REFLECT) && len < 3) return FVNA_ERR_ARG;
  if ((D.bc[0] == BC_PERIODIC) != (D.bc[1] == BC_PERIODIC)) return FVNA_ERR_ARG;
  if ((D.bc[2] == BC_PERIODIC) != (D.bc[3] == BC_PERIODIC)) return FVNA_ERR_ARG;
  // a driven rule needs the border buffer fvna_init sized for that side
  const DomDev &g = c->dd[domain];
  if (bc == BC_TAYLOR && c->cfg.precision == FVNA_FP32_PERT && !g.ghost32) return FVNA_ERR_ARG;
  if (bc == BC_HIFU && side == 0) {
    if (c->cfg.precision == FVNA_FP64 && !g.drive) return FVNA_ERR_ARG;
    if (c->cfg.precision == FVNA_FP32_PERT && !g.ghost32) return FVNA_ERR_ARG;
  }
  CK(launch_set_bc(c->d_dd, domain, side, bc, c->stream));
  c->launches += 1;
  c->doms[domain].bc[side] = bc;
  c->dd[domain].bc[side] = bc;
  return FVNA_OK;
}

int fvna_run_moving(fvna_ctx *c, double t_end, long long max_steps, double t1, double vx,
                    double vy, int every, fvna_stats *stats) {
  if (!c || max_steps < 0 || every < 1) return FVNA_ERR_ARG;
  int rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  // a time limit ends the run once a domain reaches it (a later chunk would
  // no longer be limited by it)
  std::vector<char> timed(c->ndom);
  for (int d = 0; d < c->ndom; d++) timed[d] = t_end > c->h_scal[d].t;
  long long left = max_steps;
  while (left > 0) {
    const long long n = std::min<long long>(every, left);
    rc = fvna_run(c, t_end, n, nullptr);
    if (rc != FVNA_OK) break;
    left -= n;
    // h_scal holds every domain's scalars after the chunk
    bool reached = false;
    for (int d = 0; d < c->ndom; d++) {
      const DomScal &S = c->h_scal[d];
      reached |= timed[d] && !(S.t < t_end);
      if (!(S.t > t1)) continue;
      const double e = S.t - t1;
      const long long tx = (long long)std::floor(vx * e / c->cfg.dx + 0.5);
      const long long ty = (long long)std::floor(vy * e / c->cfg.dx + 0.5);
      const long long kx = tx - c->moved_x[d], ky = ty - c->moved_y[d];
      if (kx == 0 && ky == 0) continue;
      if (std::llabs(kx) >= c->doms[d].nx || std::llabs(ky) >= c->doms[d].ny) {
        rc = FVNA_ERR_ARG;   // the window would leave its whole width behind
        break;
      }
      rc = fvna_shift(c, d, (int)kx, (int)ky);
      if (rc != FVNA_OK) break;
    }
    if (rc != FVNA_OK || reached) break;
  }
  if (rc == FVNA_OK) rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  if (stats) fill_stats(c->h_scal[0], stats);
  return first_status(c);
}

int fvna_sync(fvna_ctx *c) {
  if (!c) return FVNA_ERR_ARG;
  int rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  return first_status(c);
}

int fvna_fields(fvna_ctx *c, int domain, int what, void *dst, size_t bytes, int dst_on_device) {
  if (!c || !dst || domain < 0 || domain >= c->ndom) return FVNA_ERR_ARG;
  const fvna_domain &D = c->doms[domain];
  size_t cells = (size_t)D.nx * D.ny;
  if (what == FVNA_FIELD_Q || what == FVNA_FIELD_PRESSURE) {
    size_t need = cells * sizeof(double) * (what == FVNA_FIELD_Q ? 3 : 1);
    if (bytes < need) return FVNA_ERR_ARG;
    int w = what == FVNA_FIELD_Q ? 0 : 1;
    if (dst_on_device) {
      CK(launch_export(c->cfg.precision, c->dd[domain], (double *)dst, w, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    } else {
      if (c->stage_bytes < need) {
        cudaFree(c->d_stage);
        c->d_stage = nullptr;
        c->stage_bytes = 0;
        size_t mx = 0;
        for (const auto &d : c->doms) mx = std::max(mx, (size_t)d.nx * d.ny * 3 * sizeof(double));
        CK(cudaMalloc(&c->d_stage, mx));
        c->stage_bytes = mx;
      }
      CK(launch_export(c->cfg.precision, c->dd[domain], c->d_stage, w, c->stream));
      CK(cudaMemcpyAsync(dst, c->d_stage, need, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    return FVNA_OK;
  }
  if (what == FVNA_FIELD_AXIS) {
    const size_t need = (size_t)D.nx * sizeof(double);
    if (bytes < need) return FVNA_ERR_ARG;
    double *out = dst_on_device ? (double *)dst : c->d_stage;
    if (!dst_on_device && (!c->d_stage || c->stage_bytes < need)) {
      cudaFree(c->d_stage);
      c->d_stage = nullptr;
      c->stage_bytes = 0;
      size_t mx = 0;
      for (const auto &d : c->doms) mx = std::max(mx, (size_t)d.nx * d.ny * 3 * sizeof(double));
      CK(cudaMalloc(&c->d_stage, mx));
      c->stage_bytes = mx;
      out = c->d_stage;
    }
    CK(launch_export(c->cfg.precision, c->dd[domain], out, 2, c->stream));
    if (!dst_on_device) CK(cudaMemcpyAsync(dst, out, need, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FVNA_OK;
  }
  if (what == FVNA_FIELD_CORNER) {
    // the device descriptor holds the corner (fvna_shift moves it there)
    if (bytes < 2 * sizeof(double)) return FVNA_ERR_ARG;
    DomDev g;
    CK(cudaMemcpyAsync(&g, c->d_dd + domain, sizeof g, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double xy[2] = {g.x0, g.y0};
    if (dst_on_device) CK(cudaMemcpy(dst, xy, sizeof xy, cudaMemcpyHostToDevice));
    else std::memcpy(dst, xy, sizeof xy);
    return FVNA_OK;
  }
  int rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  const DomScal &S = c->h_scal[domain];
  if (what == FVNA_FIELD_BUDGET) {
    if (bytes < 3 * sizeof(double)) return FVNA_ERR_ARG;
    if (c->cfg.precision == FVNA_FP32_PERT || c->cfg.splitting == FVNA_SPLIT_STRANG) {
      // binary32, and binary64 Strang steps (whose sweeps end after the sum
      // the x2 sweep accumulates): summed on demand from the stored state
      double b[3];
      if (c->cfg.precision == FVNA_FP32_PERT)
        CK(launch_budget_fp32(c->dd[domain], c->d_budget, c->stream));
      else
        CK(launch_budget_fp64(c->dd[domain], c->d_budget, c->stream));
      CK(cudaMemcpyAsync(b, c->d_budget, sizeof b, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (dst_on_device) CK(cudaMemcpy(dst, b, sizeof b, cudaMemcpyHostToDevice));
      else std::memcpy(dst, b, sizeof b);
      return FVNA_OK;
    }
    if (dst_on_device) CK(cudaMemcpy(dst, S.budget, 3 * sizeof(double), cudaMemcpyHostToDevice));
    else std::memcpy(dst, S.budget, 3 * sizeof(double));
    return FVNA_OK;
  }
  if (what == FVNA_FIELD_OUTFLOW) {
    if (bytes < 3 * sizeof(double)) return FVNA_ERR_ARG;
    if (dst_on_device) CK(cudaMemcpy(dst, S.outflow, 3 * sizeof(double), cudaMemcpyHostToDevice));
    else std::memcpy(dst, S.outflow, 3 * sizeof(double));
    return FVNA_OK;
  }
  if (what == FVNA_FIELD_STATS) {
    if (bytes < sizeof(fvna_stats)) return FVNA_ERR_ARG;
    fvna_stats st;
    fill_stats(S, &st);
    if (dst_on_device) CK(cudaMemcpy(dst, &st, sizeof st, cudaMemcpyHostToDevice));
    else std::memcpy(dst, &st, sizeof st);
    return FVNA_OK;
  }
  return FVNA_ERR_ARG;
}

int fvna_step_timed(fvna_ctx *c, float ms[3]) {
  if (!c || !ms) return FVNA_ERR_ARG;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < 4; i++) {
    cudaError_t e = cudaEventCreate(&ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; j++) cudaEventDestroy(ev[j]);
      return cuda_err(e);
    }
  }
  cudaError_t e = launch_prepare(c->args, -1e300, 1, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
  if (e == cudaSuccess && enqueue_drives(c, c->stream) != FVNA_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess)
    e = sweep_x(c, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
  if (e == cudaSuccess) e = sweep_y(c, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);
  if (e == cudaSuccess && c->cfg.splitting == FVNA_SPLIT_STRANG) {
    e = sweep_x(c, c->stream);
    if (e == cudaSuccess)
      e = launch_copy_back(c->args, c->cfg.precision == FVNA_FP64 ? 8 : 4, c->stream);
  }
  if (e == cudaSuccess && !c->args_y.fold_advance) e = launch_advance(c->args, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[3], c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
  for (int i = 0; i < 4; i++) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return cuda_err(e);
  c->launches += c->kernels_per_step + 1;
  int rc = read_scal(c);
  if (rc != FVNA_OK) return rc;
  return first_status(c);
}

int fvna_autotune(const fvna_config *cfg, int n, const fvna_domain *doms, const double *const *q0,
                  int q0_on_device, void *stream, int trial_steps, fvna_config *best,
                  float *ms_per_step) {
  if (!best || trial_steps < 1) return FVNA_ERR_ARG;
  int v = validate(cfg, n, doms, q0);
  if (v != FVNA_OK) return v;
  static const int TX[4] = {X32H_TILE, 16, 32, 64};
  // binary64: heights of the column tiles; binary32: heights whose marched
  // rows (tile plus the 3-row halo on both sides) fill whole 8-row chunks
  static const int TY64[5] = {8, 16, 32, 64, 128};
  static const int TY32[5] = {10, 18, 26, 34, 42};
  const int *TY = cfg->precision == FVNA_FP32_PERT ? TY32 : TY64;
  float best_ms = -1.0f;
  fvna_config winner = *cfg;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_err(ce);
  }
  int rc = FVNA_OK;
  const int ntx = cfg->precision == FVNA_FP32_PERT ? 4 : 3;
  for (int a = 0; a < ntx && rc == FVNA_OK; a++)
    for (int b = 0; b < 5 && rc == FVNA_OK; b++) {
      fvna_config trial = *cfg;
      trial.tile_x = TX[cfg->precision == FVNA_FP32_PERT ? a : a + 1];
      trial.tile_y = TY[b];
      trial.steps_per_graph = trial_steps;
      fvna_ctx *c = new (std::nothrow) fvna_ctx();
      if (!c) { rc = FVNA_ERR_OOM; break; }
      rc = init_impl(&trial, n, doms, q0, q0_on_device, stream, c);
      if (rc == FVNA_OK) rc = ensure_graph(c);
      float ms = 0.0f;
      for (int rep = 0; rep < 2 && rc == FVNA_OK; rep++) {  // warm-up, then timed
        cudaError_t e = launch_prepare(c->args, -1e300, trial_steps, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_err(e);
      }
      if (c->stream) cudaStreamSynchronize(c->stream);
      free_ctx(c);
      if (rc == FVNA_OK && (best_ms < 0.0f || ms < best_ms)) {
        best_ms = ms;
        winner = trial;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FVNA_OK) return rc;
  winner.steps_per_graph = cfg->steps_per_graph;
  *best = winner;
  if (ms_per_step) *ms_per_step = best_ms / (float)trial_steps;
  return FVNA_OK;
}

int fvna_set_correction(fvna_ctx *c, fvna_net *net, float in_scale, float out_scale, int every,
                        int edge_band) {
  if (!c || every < 1 || edge_band < 0) return FVNA_ERR_ARG;
  if (net && (c->ndom != 1 || c->cfg.precision != FVNA_FP32_PERT)) return FVNA_ERR_ARG;
  if (net && c->cfg.splitting != FVNA_SPLIT_GODUNOV) return FVNA_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  // the correction runs between the x2 sweep and the step end, so with a
  // network the step end is its own launch again
  c->kernels_per_step += (net ? 3 : 0) - (c->net ? 3 : 0);
  if (c->cfg.precision == FVNA_FP32_PERT) {
    c->kernels_per_step += (net ? 1 : 0) - (c->net ? 1 : 0);
    c->args_y.fold_advance = net ? 0 : 1;
  }
  c->net = net;
  c->net_in = in_scale;
  c->net_out = out_scale;
  c->net_every = every;
  c->net_band = edge_band;
  if (net && !c->net_h) {
    size_t pix = (size_t)c->dd[0].nx * c->dd[0].ny;
    CK(cudaMalloc(&c->net_h, 2 * pix * 32 * sizeof(__nv_bfloat16)));
  }
  return FVNA_OK;
}

int fvna_set_budgets(fvna_ctx *c, int on) {
  if (!c || (on != 0 && on != 1)) return FVNA_ERR_ARG;
  if (on) CK(launch_zero_outflow(c->args, c->stream));
  if (on != c->budgets) {
    // the step graph is captured again with (or without) the budget kernels
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->kernels_per_step += on ? (c->cfg.splitting == FVNA_SPLIT_STRANG ? 3 : 2)
                              : -(c->cfg.splitting == FVNA_SPLIT_STRANG ? 3 : 2);
    c->budgets = on;
  }
  CK(cudaStreamSynchronize(c->stream));
  return FVNA_OK;
}

long long fvna_launch_count(const fvna_ctx *c) { return c ? c->launches : 0; }

void fvna_destroy(fvna_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

int fvna_riemann(int precision, double beta, int n, const double *qL, const double *qR, double *s,
                 double *W, double *amdq, double *apdq) {
  if (precision != FVNA_FP64 && precision != FVNA_FP32_PERT) return FVNA_ERR_ARG;
  if (n < 0 || (n > 0 && (!qL || !qR || !s || !W || !amdq || !apdq))) return FVNA_ERR_ARG;
  if (n == 0) return FVNA_OK;
  double *d = nullptr;
  int *dnr = nullptr;
  size_t per = 3 + 3 + 3 + 9 + 3 + 3;
  CK(cudaMalloc(&d, sizeof(double) * per * n));
  cudaError_t e = cudaMalloc(&dnr, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_err(e);
  }
  double *dqL = d, *dqR = d + 3 * n, *ds = d + 6 * n, *dW = d + 9 * n, *dam = d + 18 * n,
         *dap = d + 21 * n;
  int nr = 0;
  e = cudaMemcpy(dqL, qL, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dqR, qR, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dnr, 0, sizeof(int));
  if (e == cudaSuccess) e = launch_riemann(precision, beta, n, dqL, dqR, ds, dW, dam, dap, dnr, 0);
  if (e == cudaSuccess) e = cudaMemcpy(s, ds, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(W, dW, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(amdq, dam, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(apdq, dap, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&nr, dnr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(dnr);
  if (e != cudaSuccess) return cuda_err(e);
  return nr ? FVNA_ERR_NONREAL : FVNA_OK;
}

}  // extern "C"
