// fvna_api3d.cu -- host runtime of the 3D entry points of include/fvna.h.
//
// A 3D context owns one domain: two sets of four SoA planes (the state and
// the swept planes, rows padded to 32 elements, each plane 256-byte
// aligned), one device scalar block (time, dt, CFL statistics, status), and
// a CUDA graph of `steps_per_graph` steps.  A step is the x1, x2 and x3
// sweeps and the source, each reading one set of planes and writing the
// other, then the dt update; the kernels of a finished run return at once,
// so a replay may overrun the end of a run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/fvna.h"
#include "fvna_launch3.h"

using namespace fvna::d3;

struct fvna3_ctx {
  fvna_config cfg;
  fvna_domain3 dom;
  Args3 base;                  // domain, scalars and parameters (no planes)
  Scal3 *d_scal = nullptr;
  Scal3 *h_scal = nullptr;
  void *d_state = nullptr;
  void *A[4] = {}, *B[4] = {};
  double *d_stage = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 32;
  int prec = 0;
  int blocks_x = 1, blocks_v = 1, blocks_e = 1;
  int kernels_per_step = 0;
  long long launches = 0;
};

namespace {

cudaError_t g_err3 = cudaSuccess;

int err3(cudaError_t e) {
  if (e == cudaSuccess) return FVNA_OK;
  g_err3 = e;
  return e == cudaErrorMemoryAllocation ? FVNA_ERR_OOM : FVNA_ERR_CUDA;
}

#define CK3(call)                              \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return err3(e_);    \
  } while (0)

int status3(int bits) {
  if (bits & S_NONREAL) return FVNA_ERR_NONREAL;
  if (bits & S_NAN) return FVNA_ERR_NAN;
  if (bits & S_CFL) return FVNA_ERR_CFL;
  return FVNA_OK;
}

bool fp64(const fvna3_ctx *c) { return c->prec == FVNA_FP64; }

Args3 with_planes(const fvna3_ctx *c, void *const in[4], void *const out[4], int dir) {
  Args3 a = c->base;
  for (int f = 0; f < 4; f++) {
    a.in[f] = in[f];
    a.out[f] = out[f];
  }
  a.dir = dir;
  return a;
}

// one step's launches; ms (or NULL) receives the device time of the x1, x2,
// x3 sweeps, the source (a copy if the enabled sub-steps end in the swept
// planes) and the dt update, from events between them
int substeps(const fvna3_ctx *c) { return c->dom.substeps ? c->dom.substeps : 15; }

int enqueue_step(fvna3_ctx *c, cudaStream_t s, cudaEvent_t *ev) {
  const int sw = substeps(c);
  void *const *cur = c->A;
  void *const *nxt = c->B;
  auto mark = [&](int k) -> cudaError_t { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
  CK3(mark(0));
  for (int d = 0; d < 3; d++) {
    if (sw & (1 << d)) {
      Args3 a = with_planes(c, cur, nxt, d);
      if (d == 0) CK3(fp64(c) ? launch3_sweep_x_64(a, c->blocks_x, s) : launch3_sweep_x_32(a, c->blocks_x, s));
      else CK3(fp64(c) ? launch3_sweep_v_64(a, c->blocks_v, s) : launch3_sweep_v_32(a, c->blocks_v, s));
      std::swap(cur, nxt);
    }
    CK3(mark(1 + d));
  }
  if (sw & 8) {
    Args3 a = with_planes(c, cur, nxt, 0);
    CK3(fp64(c) ? launch3_source_64(a, c->blocks_e, s) : launch3_source_32(a, c->blocks_e, s));
    std::swap(cur, nxt);
  }
  if (cur != c->A) {
    Args3 a = with_planes(c, cur, nxt, 0);
    CK3(fp64(c) ? launch3_copy_64(a, c->blocks_e, s) : launch3_copy_32(a, c->blocks_e, s));
  }
  CK3(mark(4));
  CK3(launch3_advance(c->base, (sw & 7) != 0, s));
  CK3(mark(5));
  return FVNA_OK;
}

int kernels_per_step(int sw) {
  int n = 1;                       // dt update
  int stages = 0;
  for (int d = 0; d < 4; d++) stages += (sw >> d) & 1;
  n += stages + (stages & 1);      // a copy back when the stages end in the swept planes
  return n;
}

int ensure_graph3(fvna3_ctx *c) {
  if (c->gexec) return FVNA_OK;
  CK3(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  int rc = FVNA_OK;
  for (int i = 0; i < c->gsteps && rc == FVNA_OK; i++) rc = enqueue_step(c, c->cap, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (rc != FVNA_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK3(e);
  c->graph = g;
  CK3(cudaGraphInstantiate(&c->gexec, g, 0));
  return FVNA_OK;
}

int read_scal3(fvna3_ctx *c) {
  CK3(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(Scal3), cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  return FVNA_OK;
}

void stats3(const Scal3 &S, fvna_stats *st) {
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
  st->status = status3(S.status);
  st->reserved = 0;
}

void free3(fvna3_ctx *c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaFree(c->d_scal);
  cudaFree(c->d_state);
  cudaFree(c->d_stage);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
}

int validate3(const fvna_config *c, const fvna_domain3 *d, const double *q0) {
  if (!c || !d || !q0) return FVNA_ERR_ARG;
  if (c->precision != FVNA_FP64 && c->precision != FVNA_FP32_PERT) return FVNA_ERR_ARG;
  if (c->geometry != FVNA_CARTESIAN) return FVNA_ERR_ARG;
  if (c->splitting != FVNA_SPLIT_GODUNOV) return FVNA_ERR_ARG;
  if (c->limiter < FVNA_LIM_MC || c->limiter > FVNA_LIM_LW) return FVNA_ERR_ARG;
  if (d->substeps < 0 || d->substeps > 15) return FVNA_ERR_ARG;
  if (!(c->dx > 0.0) || !std::isfinite(c->dx)) return FVNA_ERR_ARG;
  if (!std::isfinite(c->beta) || !(c->delta >= 0.0) || !std::isfinite(c->delta)) return FVNA_ERR_ARG;
  if (!(c->dt_fixed > 0.0) && !(c->nu_w > 0.0)) return FVNA_ERR_ARG;
  if (!(c->nu_max > 0.0)) return FVNA_ERR_ARG;
  if (c->steps_per_graph < 0 || c->steps_per_graph > 4096) return FVNA_ERR_ARG;
  if (c->tile_y != 0 && (c->tile_y < 4 || c->tile_y > 4096)) return FVNA_ERR_ARG;
  if (c->compensated != 0 && c->compensated != 1) return FVNA_ERR_ARG;
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int k = 0; k < 3; k++)
    if (n[k] < 1 || n[k] > (1 << 16)) return FVNA_ERR_ARG;
  if ((long long)d->nx * d->ny * d->nz > (1ll << 32)) return FVNA_ERR_ARG;
  for (int s = 0; s < 6; s++) {
    int b = d->bc[s];
    if (b != FVNA_BC_PERIODIC && b != FVNA_BC_EXTRAP && b != FVNA_BC_REFLECT) return FVNA_ERR_ARG;
    if (b != FVNA_BC_EXTRAP && n[s / 2] < 3) return FVNA_ERR_ARG;
  }
  for (int k = 0; k < 3; k++)
    if ((d->bc[2 * k] == FVNA_BC_PERIODIC) != (d->bc[2 * k + 1] == FVNA_BC_PERIODIC))
      return FVNA_ERR_ARG;
  if (!(d->dt0 >= 0.0) || !std::isfinite(d->t0)) return FVNA_ERR_ARG;
  return FVNA_OK;
}

int init3(const fvna_config *cfg, const fvna_domain3 *dom, const double *q0, int q0_on_device,
          void *stream, fvna3_ctx *c) {
  c->cfg = *cfg;
  c->dom = *dom;
  c->prec = cfg->precision;
  c->stream = (cudaStream_t)stream;
  c->gsteps = cfg->steps_per_graph > 0 ? cfg->steps_per_graph : 32;
  const size_t esz = fp64(c) ? 8 : 4;
  Dom3 D;
  std::memset(&D, 0, sizeof D);
  D.nx = dom->nx; D.ny = dom->ny; D.nz = dom->nz;
  D.pitch = (dom->nx + 31) / 32 * 32;
  D.plane = (long long)D.pitch * D.ny * D.nz;
  for (int s = 0; s < 6; s++) D.bc[s] = dom->bc[s];
  const size_t plane_bytes = ((size_t)D.plane * esz + 255) / 256 * 256;
  CK3(cudaMalloc(&c->d_state, 8 * plane_bytes));
  CK3(cudaMemsetAsync(c->d_state, 0, 8 * plane_bytes, c->stream));
  for (int f = 0; f < 4; f++) {
    c->A[f] = (char *)c->d_state + f * plane_bytes;
    c->B[f] = (char *)c->d_state + (4 + f) * plane_bytes;
  }
  Scal3 sc;
  std::memset(&sc, 0, sizeof sc);
  sc.t = dom->t0;
  sc.nu_min = 1e300;
  sc.done = 1;
  CK3(cudaMalloc(&c->d_scal, sizeof(Scal3)));
  CK3(cudaMemcpyAsync(c->d_scal, &sc, sizeof sc, cudaMemcpyHostToDevice, c->stream));
  CK3(cudaMallocHost(&c->h_scal, sizeof(Scal3)));

  Args3 &a = c->base;
  std::memset(&a, 0, sizeof a);
  a.d = D;
  a.S = c->d_scal;
  a.beta = cfg->beta; a.delta = cfg->delta; a.dx = cfg->dx;
  a.nu_w = cfg->nu_w; a.nu_max = cfg->nu_max; a.dt_fixed = cfg->dt_fixed;
  a.limiter = cfg->limiter;
  a.comp = !fp64(c) && cfg->compensated ? 1 : 0;
  a.tile = cfg->tile_y ? cfg->tile_y : 64;

  // persistent grids: the sweeps' tiles handed out grid-stride
  int dev = 0, sms = 0, ox = 0, ov = 0;
  CK3(cudaGetDevice(&dev));
  CK3(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (fp64(c)) occupancy3_64(cfg->limiter, 0, &ox, &ov);
  else occupancy3_32(cfg->limiter, a.comp, &ox, &ov);
  const int tx = fp64(c) ? tile_x3_64() : tile_x3_32();
  const long long xt = (long long)((D.nx + tx - 1) / tx) * D.ny * (long long)D.nz;
  const long long vt2 = (long long)((D.nx + 31) / 32) * ((D.ny + a.tile - 1) / a.tile) * D.nz;
  const long long vt3 = (long long)((D.nx + 31) / 32) * ((D.nz + a.tile - 1) / a.tile) * D.ny;
  const long long vt = std::max(vt2, vt3);
  c->blocks_x = (int)std::max<long long>(1, std::min<long long>((xt + 3) / 4,
                                                                (long long)std::max(ox, 1) * sms));
  c->blocks_v = (int)std::max<long long>(1, std::min<long long>((vt + 3) / 4,
                                                                (long long)std::max(ov, 1) * sms));
  c->blocks_e = std::max(1, std::min((int)((D.plane + 255) / 256), 16 * sms));
  c->kernels_per_step = kernels_per_step(substeps(c));

  // initial state
  const size_t bytes = (size_t)dom->nx * dom->ny * dom->nz * 4 * sizeof(double);
  const double *src = q0;
  if (!q0_on_device) {
    CK3(cudaMalloc(&c->d_stage, bytes));
    CK3(cudaMemcpyAsync(c->d_stage, q0, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->d_stage;
  }
  Args3 ai = with_planes(c, c->A, c->A, 0);
  CK3(fp64(c) ? launch3_import_64(ai, src, c->stream) : launch3_import_32(ai, src, c->stream));
  // speed pass over the initial state -> first dt (section 4)
  const int sb = std::max(1, std::min((int)((D.plane + 255) / 256), 8 * sms));
  CK3(fp64(c) ? launch3_speeds_64(ai, sb, c->stream) : launch3_speeds_32(ai, sb, c->stream));
  CK3(launch3_first_dt(c->base, dom->dt0, c->stream));
  CK3(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  CK3(cudaStreamSynchronize(c->stream));
  return FVNA_OK;
}

}  // namespace

extern "C" {

int fvna3_init(const fvna_config *cfg, const fvna_domain3 *dom, const double *q0, int q0_on_device,
               void *stream, fvna3_ctx **out) {
  if (!out) return FVNA_ERR_ARG;
  *out = nullptr;
  int v = validate3(cfg, dom, q0);
  if (v != FVNA_OK) return v;
  fvna3_ctx *c = new (std::nothrow) fvna3_ctx();
  if (!c) return FVNA_ERR_OOM;
  int rc = init3(cfg, dom, q0, q0_on_device, stream, c);
  if (rc != FVNA_OK) {
    free3(c);
    return rc;
  }
  *out = c;
  return FVNA_OK;
}

int fvna3_run(fvna3_ctx *c, double t_end, long long max_steps, fvna_stats *stats) {
  if (!c) return FVNA_ERR_ARG;
  int rc = ensure_graph3(c);
  if (rc != FVNA_OK) return rc;
  CK3(launch3_prepare(c->base, t_end, max_steps, c->stream));
  c->launches += 1;
  // replay graphs until the device says the run is done; the host reads the
  // scalars after every batch of replays (one replay when steps are few)
  long long left = max_steps;
  for (;;) {
    long long reps = std::max<long long>(1, std::min<long long>(left / c->gsteps, 8));
    for (long long i = 0; i < reps; i++) {
      CK3(cudaGraphLaunch(c->gexec, c->stream));
      c->launches += (long long)c->gsteps * c->kernels_per_step;
    }
    rc = read_scal3(c);
    if (rc != FVNA_OK) return rc;
    if (c->h_scal->done) break;
    left -= reps * c->gsteps;
    if (left <= 0) left = c->gsteps;
  }
  if (stats) stats3(*c->h_scal, stats);
  return status3(c->h_scal->status);
}

int fvna3_step_timed(fvna3_ctx *c, float ms[5]) {
  if (!c || !ms) return FVNA_ERR_ARG;
  CK3(launch3_prepare(c->base, -1e300, 1, c->stream));
  cudaEvent_t ev[6];
  for (int k = 0; k < 6; k++) CK3(cudaEventCreate(&ev[k]));
  int rc = enqueue_step(c, c->stream, ev);
  c->launches += 1 + c->kernels_per_step;
  if (rc == FVNA_OK) {
    CK3(cudaEventSynchronize(ev[5]));
    for (int k = 0; k < 5; k++) CK3(cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]));
  }
  for (int k = 0; k < 6; k++) cudaEventDestroy(ev[k]);
  if (rc != FVNA_OK) return rc;
  rc = read_scal3(c);
  if (rc != FVNA_OK) return rc;
  return status3(c->h_scal->status);
}

int fvna3_fields(fvna3_ctx *c, int what, void *dst, size_t bytes, int dst_on_device) {
  if (!c || !dst) return FVNA_ERR_ARG;
  const size_t n = (size_t)c->dom.nx * c->dom.ny * c->dom.nz;
  if (what == FVNA_FIELD_STATS) {
    if (bytes < sizeof(fvna_stats)) return FVNA_ERR_ARG;
    int rc = read_scal3(c);
    if (rc != FVNA_OK) return rc;
    fvna_stats st;
    stats3(*c->h_scal, &st);
    if (dst_on_device) CK3(cudaMemcpy(dst, &st, sizeof st, cudaMemcpyHostToDevice));
    else std::memcpy(dst, &st, sizeof st);
    return FVNA_OK;
  }
  if (what != FVNA_FIELD_Q && what != FVNA_FIELD_PRESSURE) return FVNA_ERR_ARG;
  const size_t need = (what == FVNA_FIELD_Q ? 4 : 1) * n * sizeof(double);
  if (bytes < need) return FVNA_ERR_ARG;
  double *out = (double *)dst;
  double *tmp = nullptr;
  if (!dst_on_device) {
    CK3(cudaMalloc(&tmp, need));
    out = tmp;
  }
  Args3 a = with_planes(c, c->A, c->A, 0);
  cudaError_t e = fp64(c) ? launch3_export_64(a, out, what == FVNA_FIELD_Q ? 0 : 1, c->stream)
                          : launch3_export_32(a, out, what == FVNA_FIELD_Q ? 0 : 1, c->stream);
  if (e == cudaSuccess && tmp)
    e = cudaMemcpyAsync(dst, tmp, need, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (tmp) cudaFree(tmp);
  return err3(e);
}

long long fvna3_launch_count(const fvna3_ctx *c) { return c ? c->launches : 0; }

void fvna3_destroy(fvna3_ctx *c) { free3(c); }

}  // extern "C"
