// fvna_sweeps32.cuh -- the binary32 sweep kernels (perturbation variables,
// arXiv 1311.3004 section 3 with the splitting of section 3.3).
//
//   k_sweep_x32  x1 sweep.  One warp (one CTA) owns a tile of 32 rows x 2 SW
//                cells.  TMA brings in the two SW-wide halves of the tile
//                (swizzled, so each lane reads 16 bytes of its own row
//                without bank conflicts) and the 4-column halo boxes on both
//                sides; each lane marches its row's two halves at once as a
//                pair of lines, writes the new cells back in place, and TMA
//                stores the halves into the swept planes.
//   k_sweep_y32  x2 sweep fused with the source sub-step.  One warp owns 60
//                columns and tile_y rows; each lane marches two adjacent
//                columns as a pair (one 8-byte shared-memory read per field
//                and row).  Rows arrive in chunks of 8 through a two-stage TMA
//                ring; the source is applied one row behind the
//                sweep, with the x1 neighbours taken from the adjacent lanes
//                by shuffles, and the result is stored with coalesced 8-byte
//                stores.
// Both sweeps take every face as subsonic (no per-face branch); a tile that
// met another face is marched again with the general split: at once by the
// same warp in the x1 sweep, by a second kernel in the x2 sweep.
// Interior tiles run without any border logic; tiles that touch a domain
// border (or a ragged edge) take the same code with per-cell border rules
// and per-face accounting masks.  Analytic border values come precomputed
// from the ghost ring (k_ghost32), so the border path stays light.
#pragma once

#include "fvna_step.cuh"
#include "fvna_sweeps.cuh"
#include "fvna_x2.cuh"

namespace fvna {

constexpr int X32_ROWS = 32;
// resident x1-sweep warps per SM the register allocator plans for: none (the
// compiler takes 254 registers, no spills).  12 (168 registers, the general
// split out of line, 12 warps per SM for 32-cell tiles) measured no faster:
// 42.3 us against 40.8 us on the 2048^2 pulse.
#ifndef X32_MINBLOCKS
#define X32_MINBLOCKS 1
#endif
#ifndef FVNA_Y_UNROLL
#define FVNA_Y_UNROLL 2   // rows of the x2 sweep's plain loop unrolled together (measured best)
#endif
#ifndef FVNA_Y32_STAGES
#define FVNA_Y32_STAGES 2
#endif
constexpr int Y32_STAGES = FVNA_Y32_STAGES;
// resident x2-sweep warps per SM the register allocator plans for (the
// shared-memory ring allows 11).  Interior tiles alone fit 128 registers
// (16 warps per SM), but a kernel of those alone measured 42 us for 93 % of
// the 2048^2 pulse's tiles and left the border tiles, whose general path
// waits on global loads of ghost cells row after row, 28 us in a second
// kernel; in one kernel they start first and overlap the interior ones.
#ifndef Y32_MINBLOCKS
#define Y32_MINBLOCKS 11
#endif
constexpr int Y32_STAGE_BYTES = 3 * x2::YRB * x2::YBOX * 4;

__host__ __device__ constexpr int x32_smem_bytes(int sw) {
  return 1024 + 6 * X32_ROWS * sw * 4 + 6 * X32_ROWS * 16 + 64;
}
__host__ __device__ constexpr int y32_smem_bytes() {
  return 128 + Y32_STAGES * Y32_STAGE_BYTES + 64;
}
namespace x2 {

// Self-checking build (FVNA_CHECK=1): every global index of the border
// rules and of the x2 sweep's stores is checked; the first bad one is
// recorded (code << 48 | index) and the access skipped.
#ifndef FVNA_CHECK
#define FVNA_CHECK 0
#endif
#if FVNA_CHECK
static __device__ unsigned long long g_check_word = 0ull;
__device__ __forceinline__ bool chk(bool ok, int code, long long idx) {
  if (!ok) atomicCAS(&g_check_word, 0ull, ((unsigned long long)code << 48) |
                                          ((unsigned long long)idx & 0xffffffffffffull));
  return ok;
}
#else
__device__ __forceinline__ bool chk(bool ok, int, long long) { return true; }
#endif

__device__ __forceinline__ float comp(const float4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// Driven borders in binary32.  The analytic border values of a step (eq.
// OurTaylorS, eq. hifuBC) are evaluated once per step in binary64 by
// k_ghost32 into the domain's ghost ring; the sweeps only read them.  Ring
// layout (3 planes of ghost_ring_size values): x1 ghosts, columns -3..-1 and
// nx..nx+2 (k = 0..5) for rows -3..ny+2; then x2 ghosts, rows -3..-1 and
// ny..ny+2 (k = 0..5) for columns -3..nx+2.  NaN marks a ghost cell that is
// not driven (a HIFU border outside the aperture).
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t ghost_ring_size(int nx, int ny) {
  return 6 * (size_t)(ny + 6) + 6 * (size_t)(nx + 6);
}
// (indices clamped into the ring: a tile's halo may reach rows beyond
// ny + 2, whose values never reach a stored cell)
__device__ __forceinline__ size_t ring_x(const DomDev &D, int gx, int gy) {
  int k = gx < 0 ? gx + 3 : gx - D.nx + 3;
  k = min(max(k, 0), 5);
  gy = min(max(gy, -3), D.ny + 2);
  return (size_t)k * (D.ny + 6) + (gy + 3);
}
__device__ __forceinline__ size_t ring_y(const DomDev &D, int cx, int gy) {
  int k = gy < 0 ? gy + 3 : gy - D.ny + 3;
  k = min(max(k, 0), 5);
  cx = min(max(cx, -3), D.nx + 2);
  return 6 * (size_t)(D.ny + 6) + (size_t)k * (D.nx + 6) + (cx + 3);
}
__device__ __forceinline__ bool ring_get(const DomDev &D, size_t o, float v[3]) {
  const float *R = (const float *)D.ghost32;
  const size_t n = ghost_ring_size(D.nx, D.ny);
  if (!chk(R != nullptr && o < n, 1, (long long)o)) {
    v[0] = v[1] = v[2] = 0.f;
    return true;
  }
  v[0] = R[o];
  v[1] = R[n + o];
  v[2] = R[2 * n + o];
  return v[0] == v[0];
}

// The border rules of load_mapped (fvna_sweeps.cuh) with the analytic values
// taken from the ghost ring: value of cell (gx, gy), -3 <= gx, gy, with
// every index outside the domain mapped.
__device__ __forceinline__ void load32(const DomDev &D, const float *const q[3], int gx, int gy,
                                       float out[3]) {
  const int nx = D.nx, ny = D.ny;
  bool flipx = false, flipy = false;
  int cx = gx, cy = gy;
  if (gx < 0 || gx >= nx) {
    if (gx > nx + HALO_Y - 1) gx = nx + HALO_Y - 1;
    int side = gx < 0 ? 0 : 1;
    int bc = D.bc[side];
    if ((bc == BC_TAYLOR || (bc == BC_HIFU && side == 0)) && ring_get(D, ring_x(D, gx, gy), out))
      return;
    if (bc == BC_PERIODIC) cx = side == 0 ? gx + nx : gx - nx;
    else if (bc == BC_REFLECT) { cx = side == 0 ? -1 - gx : 2 * nx - 1 - gx; flipx = true; }
    else cx = side == 0 ? 0 : nx - 1;
  }
  if (gy < 0 || gy >= ny) {
    if (gy > ny + HALO_Y - 1) gy = ny + HALO_Y - 1;
    int side = gy < 0 ? 0 : 1;
    int bc = D.bc[2 + side];
    if (bc == BC_TAYLOR) {
      ring_get(D, ring_y(D, cx, gy), out);
      if (flipx) out[1] = -out[1];
      return;
    }
    if (bc == BC_PERIODIC) cy = side == 0 ? gy + ny : gy - ny;
    else if (bc == BC_REFLECT) { cy = side == 0 ? -1 - gy : 2 * ny - 1 - gy; flipy = true; }
    else cy = side == 0 ? 0 : ny - 1;
  }
  if (!chk(cx >= 0 && cx < nx && cy >= 0 && cy < ny, 2, (long long)cy * 65536 + cx)) {
    out[0] = out[1] = out[2] = 0.f;
    return;
  }
  size_t off = (size_t)cy * D.pitch + cx;
  float v0 = q[0][off], v1 = q[1][off], v2 = q[2][off];
  out[0] = v0;
  out[1] = flipx ? -v1 : v1;
  out[2] = flipy ? -v2 : v2;
}
// Is the x1 ghost cell (gx, gy) driven?  (x_driven of fvna_sweeps.cuh)
__device__ __forceinline__ bool xdriven32(const DomDev &D, int gx, int gy) {
  if (gx >= 0 && gx < D.nx) return false;
  int side = gx < 0 ? 0 : 1;
  int bc = D.bc[side];
  if (bc == BC_TAYLOR) return true;
  if (bc == BC_HIFU && side == 0) return ((const float *)D.ghost32)[ring_x(D, gx, gy)] ==
                                          ((const float *)D.ghost32)[ring_x(D, gx, gy)];
  return false;
}

// Swizzled byte offset of (row r, column c) in a box whose rows are RB bytes
// (TMA swizzle of span RB: the 16-byte chunk index is XORed with address
// bits 7 and up; the buffer is 1024-byte aligned).
template <int RB> __device__ __forceinline__ unsigned swz(unsigned r, unsigned c) {
  unsigned o = r * RB + c * 4;
  return o ^ ((o >> 3) & (unsigned)((RB / 16 - 1) << 4));
}

// Dynamic tile schedule: the warps of a sweep take tiles from a shared
// counter (the host lists the slow border tiles first, so they start
// early).  Each sweep resets the other sweep's counter, which is idle then.
__device__ __forceinline__ int take_tile(unsigned *ctr, int lane) {
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(ctr, 1u);
  return (int)__shfl_sync(0xffffffffu, t, 0);
}
// the same in two halves: the atomic is issued when a tile starts and its
// result broadcast when the tile ends, so the march hides its latency
__device__ __forceinline__ unsigned take_tile_issue(unsigned *ctr, int lane) {
  return lane == 0 ? atomicAdd(ctr, 1u) : 0u;
}
__device__ __forceinline__ int take_tile_collect(unsigned t) {
  return (int)__shfl_sync(0xffffffffu, t, 0);
}

// error exit of a failed wait: flag the domain, let the copy land (default
// limit, whatever the first wait's was), stop
__device__ __forceinline__ void wait_failed(DomScal *S, uint64_t *bar, unsigned parity, int lane) {
  if (lane == 0) atomicOr(&S->status_bits, ST_TIMEOUT);
  mbar_wait(bar, parity);
}

// warp-wide statistics of a tile into the domain scalars
__device__ __forceinline__ void flush_acc(const Acc &a, DomScal *S, int lane) {
  unsigned b = max(SpeedBits<float>::bits(a.smax.x), SpeedBits<float>::bits(a.smax.y));
  if (a.smax.x != a.smax.x || a.smax.y != a.smax.y) b = 0x7fc00000u;
  b = SpeedBits<float>::warp_max(b);
  bool nr = fminf(a.c2min.x, a.c2min.y) < 0.f;
  nr = __any_sync(0xffffffffu, nr);
  if (lane == 0) {
    if (b) atomic_max_speed(&S->smax_bits, SpeedBits<float>::value(b));
    if (nr) atomicOr(&S->status_bits, ST_NONREAL);
  }
}

// ---------------------------------------------------------------------------
// x1 sweep
// ---------------------------------------------------------------------------
// Returns false (and leaves the statistics alone) when SPEC marched a face
// that was not subsonic: the tile must then be reloaded and redone.
template <int SW, int LIM, bool COMP, bool BORDER, bool SPEC>
__device__ __forceinline__ bool x32_tile(const StepArgs &A, const DomDev &D, DomScal *S,
                                         unsigned char *mainb, unsigned char *halo, int x0, int y0,
                                         int lane) {
  constexpr int RB = SW * 4;
  constexpr int BOX = X32_ROWS * RB;
  constexpr int HB = X32_ROWS * 16;
  const int r = lane, gy = y0 + r;
  const int nx = D.nx;
  const bool row_ok = gy < D.ny;
  if (BORDER && row_ok) {
    // ghost cells of this row, mapped by the border rules of section 4
    const float *qi[3] = {(const float *)D.qa[0], (const float *)D.qa[1], (const float *)D.qa[2]};
    for (int g = 0; g < 4; g++) {
      int gx = g < 2 ? g - 2 : nx + g - 2;
      if (g < 2 && x0 != 0) continue;
      int p = gx - (x0 - 4);
      if (p < 2 || p >= 2 * SW + 6) continue;
      float v[3];
      load32(D, qi, gx, gy, v);
      for (int f = 0; f < 3; f++) {
        float *dst;
        if (p < 4) dst = (float *)(halo + 2 * f * HB + r * 16 + p * 4);
        else if (p < 4 + 2 * SW) {
          int q = p - 4, seg = q / SW;
          dst = (float *)(mainb + (2 * f + seg) * BOX + swz<RB>(r, q - seg * SW));
        } else dst = (float *)(halo + (2 * f + 1) * HB + r * 16 + (p - 4 - 2 * SW) * 4);
        *dst = v[f];
      }
    }
  }
  March<LIM, COMP, SPEC> m;
  // dt/dx, halved (exactly) for the two x1 sweeps of a Strang step
  m.init((float)A.beta, A.x_half ? 0.5f * S->lam32 : S->lam32);
  // cells x0+SW, x0+SW+1 (right neighbours of the first half) before the
  // second half overwrites them
  float2 rA[3];
  for (int f = 0; f < 3; f++)
    rA[f] = *(const float2 *)(mainb + (2 * f + 1) * BOX + swz<RB>(r, 0));
  // accounting masks of face j of each half (border tiles): |s| over the
  // domain's faces 0..nx, the non-real test over faces -1..nx+1
  auto mask = [&](int j, bool &sx, bool &sy, bool &nx_, bool &ny_) {
    int ga = x0 - 2 + j, gb = x0 + SW - 2 + j;
    sx = row_ok && ga >= 0 && ga <= nx;
    sy = row_ok && gb >= 0 && gb <= nx;
    nx_ = row_ok && ga >= -1 && ga <= nx + 1;
    ny_ = row_ok && gb >= -1 && gb <= nx + 1;
  };
  bool sx = true, sy = true, nx_ = true, ny_ = true;
  Cell out;
  // cells j = 0, 1: halo of the first half, last two cells of the first
  // half for the second
  {
    float2 ha[3], hb[3];
    for (int f = 0; f < 3; f++) {
      ha[f] = *(const float2 *)(halo + 2 * f * HB + r * 16 + 8);
      hb[f] = *(const float2 *)(mainb + 2 * f * BOX + swz<RB>(r, SW - 2));
    }
    Cell q0, q1;
    q0.a = make_float2(ha[0].x, hb[0].x); q0.b = make_float2(ha[1].x, hb[1].x);
    q0.c = make_float2(ha[2].x, hb[2].x);
    q1.a = make_float2(ha[0].y, hb[0].y); q1.b = make_float2(ha[1].y, hb[1].y);
    q1.c = make_float2(ha[2].y, hb[2].y);
    m.template push<false>(0, q0, out, true, true, true, true, false);
    if (BORDER) mask(1, sx, sy, nx_, ny_);
    m.template push<BORDER>(1, q1, out, sx, sy, nx_, ny_, false);
  }
  // updated cells wait in registers until four consecutive columns of a
  // half are complete (one 16-byte store per field and half)
  Cell h0, h1, n0, n1;
  auto put = [&](int k) {  // columns 4k..4k+3 = h0, h1, n0, n1
    *(float4 *)(mainb + 0 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.a.x, h1.a.x, n0.a.x, n1.a.x);
    *(float4 *)(mainb + 1 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.a.y, h1.a.y, n0.a.y, n1.a.y);
    *(float4 *)(mainb + 2 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.b.x, h1.b.x, n0.b.x, n1.b.x);
    *(float4 *)(mainb + 3 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.b.y, h1.b.y, n0.b.y, n1.b.y);
    *(float4 *)(mainb + 4 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.c.x, h1.c.x, n0.c.x, n1.c.x);
    *(float4 *)(mainb + 5 * BOX + swz<RB>(r, 4 * k)) = make_float4(h0.c.y, h1.c.y, n0.c.y, n1.c.y);
  };
  auto chunk_cell = [&](const float4 (&va)[3], const float4 (&vb)[3], int i) {
    Cell q;
    q.a = make_float2(comp(va[0], i), comp(vb[0], i));
    q.b = make_float2(comp(va[1], i), comp(vb[1], i));
    q.c = make_float2(comp(va[2], i), comp(vb[2], i));
    return q;
  };
  // chunk 0: cells j = 2..5, updates of columns 0 and 1
  {
    float4 va[3], vb[3];
    for (int f = 0; f < 3; f++) {
      va[f] = *(const float4 *)(mainb + 2 * f * BOX + swz<RB>(r, 0));
      vb[f] = *(const float4 *)(mainb + (2 * f + 1) * BOX + swz<RB>(r, 0));
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (BORDER) mask(2 + i, sx, sy, nx_, ny_);
      m.template push<BORDER>(2 + i, chunk_cell(va, vb, i), out, sx, sy, nx_, ny_, false);
      if (i == 2) h0 = out;
      if (i == 3) h1 = out;
    }
  }
  // chunks 1..SW/4-1, the next chunk's shared-memory reads issued one chunk
  // ahead
  float4 va[3], vb[3];
  for (int f = 0; f < 3; f++) {
    va[f] = *(const float4 *)(mainb + 2 * f * BOX + swz<RB>(r, 4));
    vb[f] = *(const float4 *)(mainb + (2 * f + 1) * BOX + swz<RB>(r, 4));
  }
#pragma unroll 1
  for (int k = 1; k < SW / 4; k++) {
    float4 ca_[3], cb_[3];
    for (int f = 0; f < 3; f++) {
      ca_[f] = va[f];
      cb_[f] = vb[f];
    }
    if (k + 1 < SW / 4)
      for (int f = 0; f < 3; f++) {
        va[f] = *(const float4 *)(mainb + 2 * f * BOX + swz<RB>(r, 4 * k + 4));
        vb[f] = *(const float4 *)(mainb + (2 * f + 1) * BOX + swz<RB>(r, 4 * k + 4));
      }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      int j = 2 + 4 * k + i;
      if (BORDER) mask(j, sx, sy, nx_, ny_);
      out = m.template step<BORDER>(chunk_cell(ca_, cb_, i), sx, sy, nx_, ny_, false);
      if (i == 0) n0 = out;
      if (i == 1) {
        n1 = out;
        put(k - 1);
      }
      if (i == 2) h0 = out;
      if (i == 3) h1 = out;
    }
  }
  // cells j = SW+2, SW+3: first two cells of the second half (read above)
  // for the first, the right halo for the second
  {
    float2 hr[3];
    for (int f = 0; f < 3; f++) hr[f] = *(const float2 *)(halo + (2 * f + 1) * HB + r * 16);
    Cell q0, q1;
    q0.a = make_float2(rA[0].x, hr[0].x); q0.b = make_float2(rA[1].x, hr[1].x);
    q0.c = make_float2(rA[2].x, hr[2].x);
    q1.a = make_float2(rA[0].y, hr[0].y); q1.b = make_float2(rA[1].y, hr[1].y);
    q1.c = make_float2(rA[2].y, hr[2].y);
    if (BORDER) mask(SW + 2, sx, sy, nx_, ny_);
    n0 = m.template step<BORDER>(q0, sx, sy, nx_, ny_, false);
    if (BORDER) mask(SW + 3, sx, sy, nx_, ny_);
    n1 = m.template step<BORDER>(q1, sx, sy, nx_, ny_, false);
    put(SW / 4 - 1);
  }
  fence_async();
  if (SPEC && !spec_held(m.acc)) return false;
  flush_acc(m.acc, S, lane);
  return true;
}

}  // namespace x2

// A tile whose speculative march met a face that is not subsonic is loaded
// again and marched with the general split by the same warp, before its
// store: its result depends only on the state planes, which no warp of the
// sweep writes.
template <int SW, int LIM, bool COMP>
__global__ void __launch_bounds__(32, X32_MINBLOCKS) k_sweep_x32(StepArgs A) {
  using namespace x2;
  constexpr int BOX = X32_ROWS * SW * 4;
  constexpr int HB = X32_ROWS * 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *mainb =
      (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *halo = mainb + 6 * BOX;
  uint64_t *bar = (uint64_t *)(halo + 6 * HB);
  const int lane = threadIdx.x;
  const Maps *maps = (const Maps *)A.tmaps;
  if (lane == 0) mbar_init(bar, 1);
  griddep_wait();
  if (blockIdx.x == 0 && lane == 0) {
    A.counters[1] = 0u;         // the x2 sweep's tile counter
    A.redo[1] = 0;              // the x2 sweep's list, empty for this step
  }
  __syncwarp();
  unsigned phase = 0;
  const bool xsweep = (A.sweeps & 1) != 0;
  const int nt = A.ntiles;
  // the tile's boxes: two swizzled halves and the halo columns on both sides
  auto load = [&](const Maps &M, int x0, int y0) {
    mbar_expect_tx(bar, 6 * BOX + 6 * HB);
    for (int f = 0; f < 3; f++) {
      tma_load(mainb + 2 * f * BOX, &M.xin[f], x0, y0, bar);
      tma_load(mainb + (2 * f + 1) * BOX, &M.xin[f], x0 + SW, y0, bar);
      tma_load(halo + 2 * f * HB, &M.xhalo[f], x0 - 4, y0, bar);
      tma_load(halo + (2 * f + 1) * HB, &M.xhalo[f], x0 + 2 * SW, y0, bar);
    }
  };
  int it = take_tile(&A.counters[0], lane);
  Tile tl = it < nt ? A.tiles[it] : Tile{0, 0, 0, 0};
  while (it < nt) {
    const unsigned tn = take_tile_issue(&A.counters[0], lane);
    const DomDev &D = A.doms[tl.dom];
    DomScal *S = A.scal + tl.dom;
    if (S->done) {
      it = take_tile_collect(tn);
      if (it < nt) tl = A.tiles[it];
      continue;
    }
    const Maps &M = maps[tl.dom];
    const int x0 = tl.x0, y0 = tl.y0;
    if (lane == 0) {
      bulk_wait_read();  // the previous tile's stores have read the buffers
      load(M, x0, y0);
    }
    bool ok = __all_sync(0xffffffffu, mbar_wait(bar, phase, A.wait_polls));
    if (!ok) {
      wait_failed(S, bar, phase, lane);
      break;
    }
    phase ^= 1;
    it = take_tile_collect(tn);
    if (it < nt) tl = A.tiles[it];
    if (xsweep) {
      bool sub = (x0 == 0 || x0 + 2 * SW + 2 > D.nx || y0 + X32_ROWS > D.ny)
                     ? x2::x32_tile<SW, LIM, COMP, true, true>(A, D, S, mainb, halo, x0, y0, lane)
                     : x2::x32_tile<SW, LIM, COMP, false, true>(A, D, S, mainb, halo, x0, y0,
                                                                lane);
      if (!sub) {
        // the march wrote into the tile: load it again, general split
        __syncwarp();
        if (lane == 0) load(M, x0, y0);
        if (!__all_sync(0xffffffffu, mbar_wait(bar, phase, A.wait_polls))) {
          wait_failed(S, bar, phase, lane);
          break;
        }
        phase ^= 1;
        x2::x32_tile<SW, LIM, COMP, true, false>(A, D, S, mainb, halo, x0, y0, lane);
      }
    }
    __syncwarp();
    if (lane == 0) {
      for (int f = 0; f < 3; f++) {
        tma_store(&M.xout[f], x0, y0, mainb + 2 * f * BOX);
        tma_store(&M.xout[f], x0 + SW, y0, mainb + (2 * f + 1) * BOX);
      }
      bulk_commit();
    }
  }
  griddep_launch();
  if (lane == 0) bulk_wait();
}

// ---------------------------------------------------------------------------
// x2 sweep + source
// ---------------------------------------------------------------------------
namespace x2 {

// Per-component column data of a lane in a border tile.
struct YCol {
  int gx;        // marched column (clamped to nx on the right, as a duplicate ghost)
  int col;       // column read for rows inside the domain
  bool inside;   // 0 <= gx < nx
  bool plain;    // rows inside the domain read column col unchanged
  bool xdrv;     // driven ghost column (analytic values replace the swept ones)
  bool upd;      // updated and accounted column of this tile
};

__device__ __forceinline__ YCol ycol(const DomDev &D, int gx, int x0, int lane) {
  YCol c;
  const int nx = D.nx;
  c.upd = lane >= 1 && lane <= 30 && gx >= x0 && gx < nx;
  if (gx > nx) gx = nx;
  c.gx = gx;
  c.col = gx;
  c.inside = gx >= 0 && gx < nx;
  c.plain = true;
  c.xdrv = false;
  if (!c.inside) {
    int side = gx < 0 ? 0 : 1;
    int bc = D.bc[side];
    if (bc == BC_PERIODIC) c.col = side == 0 ? gx + nx : gx - nx;
    else if (bc == BC_REFLECT) { c.col = side == 0 ? 0 : nx - 1; c.plain = false; }
    else if (bc == BC_TAYLOR) { c.col = side == 0 ? 0 : nx - 1; c.xdrv = true; }
    else if (bc == BC_HIFU && side == 0) { c.col = 0; c.xdrv = true; }
    else c.col = side == 0 ? 0 : nx - 1;
  }
  return c;
}

// value of (gx, gy) for a border tile: shared memory for inside cells, the
// border rules for the rest (the same reads as the binary64 sweep)
__device__ __forceinline__ void ycell(const DomDev &D, const YCol &c, int gy,
                                      const float *const q[3], float s0, float s1, float s2,
                                      float v[3]) {
  if (c.inside && gy >= 0 && gy < D.ny) {
    v[0] = s0; v[1] = s1; v[2] = s2;
    return;
  }
  if (c.plain && gy >= 0 && gy < D.ny && chk(c.col >= 0 && c.col < D.nx, 3, c.col)) {
    size_t off = (size_t)gy * D.pitch + c.col;
    v[0] = q[0][off]; v[1] = q[1][off]; v[2] = q[2][off];
    return;
  }
  load32(D, q, c.gx, gy, v);
}

// Source sub-step, one row behind the x2 sweep (the binary32 counterpart of
// the binary64 sink): holds the post-sweep row e-1 and the velocities z of
// rows e-1 and e-2.
struct YSrc {
  V qp0, qp1, qp2, zp2, zp3, zpp2, zpp3;
};

template <bool BORDER>
__device__ __forceinline__ void ysink(YSrc &s, const StepArgs &A, const DomDev &D, int x0, int y0,
                                      int TY, int lane, int e, V q0, V q1, V q2, bool source,
                                      bool axi, float coef, float dt32, const YCol &ca,
                                      const YCol &cb, float *const qo[3]) {
  const int ny = D.ny;
  if (BORDER) {
    // driven ghost columns: analytic values replace the swept ones
    for (int k = 0; k < 2; k++) {
      const YCol &c = k ? cb : ca;
      if (c.xdrv && e >= 0 && e < ny && xdriven32(D, c.gx, e)) {
        float v[3];
        ring_get(D, ring_x(D, c.gx, e), v);
        if (k) { q0.y = v[0]; q1.y = v[1]; q2.y = v[2]; }
        else { q0.x = v[0]; q1.x = v[1]; q2.x = v[2]; }
      }
    }
    if (e == ny) {  // x2-high ghost row from the post-sweep row ny-1
      int bc = D.bc[3];
      if (bc == BC_EXTRAP || bc == BC_HIFU) { q0 = s.qp0; q1 = s.qp1; q2 = s.qp2; }
      else if (bc == BC_REFLECT) { q0 = s.qp0; q1 = s.qp1; q2 = make_float2(-s.qp2.x, -s.qp2.y); }
      else if (bc == BC_TAYLOR) {
        for (int k = 0; k < 2; k++) {
          float v[3];
          ring_get(D, ring_y(D, k ? cb.gx : ca.gx, e), v);
          if (k) { q0.y = v[0]; q1.y = v[1]; q2.y = v[2]; }
          else { q0.x = v[0]; q1.x = v[1]; q2.x = v[2]; }
        }
      }
    }
  }
  Cell qc;
  qc.a = q0; qc.b = q1; qc.c = q2;
  V z2, z3;
  zof(qc, z2, z3);
  if (BORDER && e == 0 && y0 == 0) {  // x2-low ghost row from the post-sweep row 0
    int bc = D.bc[2];
    if (bc == BC_EXTRAP || bc == BC_HIFU) { s.zp2 = z2; s.zp3 = z3; }
    else if (bc == BC_REFLECT) { s.zp2 = z2; s.zp3 = make_float2(-z3.x, -z3.y); }
    else if (bc == BC_TAYLOR) {
      for (int k = 0; k < 2; k++) {
        float v[3];
        ring_get(D, ring_y(D, k ? cb.gx : ca.gx, -1), v);
        float r = 1.f / (1.f + v[0]);
        if (k) { s.zp2.y = v[1] * r; s.zp3.y = v[2] * r; }
        else { s.zp2.x = v[1] * r; s.zp3.x = v[2] * r; }
      }
    }
  }
  // source on row e-1: x1 neighbours of column A are (lane-1).B and B; of
  // column B, A and (lane+1).A
  const int er = e - 1;
  float w2 = __shfl_up_sync(0xffffffffu, s.zp2.y, 1);
  float e2 = __shfl_down_sync(0xffffffffu, s.zp2.x, 1);
  float w3 = __shfl_up_sync(0xffffffffu, s.zp3.y, 1);
  float e3 = __shfl_down_sync(0xffffffffu, s.zp3.x, 1);
  bool store_row = er >= y0 && er < y0 + TY && (!BORDER || er < ny);
  if (store_row) {
    V o0 = s.qp0, o1 = s.qp1, o2 = s.qp2;
    if (source) {
      V W2 = make_float2(w2, s.zp2.x), E2 = make_float2(s.zp2.y, e2);
      V W3 = make_float2(w3, s.zp3.x), E3 = make_float2(s.zp3.y, e3);
      V L2 = fma(s.zp2, vs(-4.f), add(add(W2, E2), add(s.zpp2, z2)));
      V L3 = fma(s.zp3, vs(-4.f), add(add(W3, E3), add(s.zpp3, z3)));
      if (!axi) {
        o1 = fma(vs(coef), L2, o1);
        o2 = fma(vs(coef), L3, o2);
      } else {
        float r = (float)D.y0 + ((float)er + 0.5f) * (float)A.dx;
        float rr = 1.f / r;
        V hdr = vs((float)A.dx / (2.f * r));
        V ddr = vs((float)A.dx * (float)A.dx * rr * rr);
        L2 = fma(sub(z2, s.zpp2), hdr, L2);
        L3 = sub(fma(sub(z3, s.zpp3), hdr, L3), mul(s.zp3, ddr));
        V g1 = mul(s.qp2, vs(rr));
        V g2 = mul(mul(s.zp2, s.zp3), vs(rr));
        V g3 = mul(mul(s.zp3, s.zp3), vs(rr));
        V ndt = vs(-dt32);
        o0 = fma(ndt, g1, o0);
        o1 = fma(ndt, g2, fma(vs(coef), L2, o1));
        o2 = fma(ndt, g3, fma(vs(coef), L3, o2));
      }
    }
    size_t off = (size_t)er * D.pitch + (x0 - 2 + 2 * lane);
    if (!BORDER) {
      if (lane >= 1 && lane <= 30) {
        *(float2 *)(qo[0] + off) = o0;
        *(float2 *)(qo[1] + off) = o1;
        *(float2 *)(qo[2] + off) = o2;
      }
    } else if (ca.upd && cb.upd) {
      *(float2 *)(qo[0] + off) = o0;
      *(float2 *)(qo[1] + off) = o1;
      *(float2 *)(qo[2] + off) = o2;
    } else if (ca.upd) {
      qo[0][off] = o0.x; qo[1][off] = o1.x; qo[2][off] = o2.x;
    } else if (cb.upd) {
      qo[0][off + 1] = o0.y; qo[1][off + 1] = o1.y; qo[2][off + 1] = o2.y;
    }
  }
  s.qp0 = q0; s.qp1 = q1; s.qp2 = q2;
  s.zpp2 = s.zp2; s.zpp3 = s.zp3;
  s.zp2 = z2; s.zp3 = z3;
}

// Returns 0 when done, 1 when a wait timed out, 2 when SPEC marched a face
// that was not subsonic (the tile must be redone with SPEC off; its rows
// were stored and will be stored again).
template <int LIM, bool COMP, bool SPEC>
__device__ __forceinline__ int y32_tile(const StepArgs &A, const DomDev &D, DomScal *S,
                                        const Maps &M, unsigned char *ring, uint64_t *bars,
                                        unsigned &used, int x0, int y0, int TY, int lane) {
  const int nrows = TY + 2 * HALO_Y;
  const int nch = (nrows + YRB - 1) / YRB;
  const unsigned base = used;
  const bool ysweep = (A.sweeps & 2) != 0;
  const bool source = (A.sweeps & 4) != 0;
  const bool axi = A.geometry == 1;
  const float coef = S->coef32, dt32 = S->dt32;
  float *qo[3] = {(float *)D.qa[0], (float *)D.qa[1], (float *)D.qa[2]};
  const float *qi[3] = {(const float *)D.qb[0], (const float *)D.qb[1], (const float *)D.qb[2]};
  auto issue = [&](int c) {
    unsigned s = (base + c) % Y32_STAGES;
    unsigned char *st = ring + s * Y32_STAGE_BYTES;
    mbar_expect_tx(&bars[s], Y32_STAGE_BYTES);
    for (int f = 0; f < 3; f++)
      tma_load(st + f * (YRB * YBOX * 4), &M.yin[f], x0 - 4, y0 - HALO_Y + c * YRB, &bars[s]);
  };
  if (lane == 0)
    for (int c = 0; c < nch && c < Y32_STAGES; c++) issue(c);
  used += nch;

  const YCol ca = ycol(D, x0 - 2 + 2 * lane, x0, lane);
  const YCol cb = ycol(D, x0 - 1 + 2 * lane, x0, lane);
  // accounting ranges (faces j, local): |s| over faces y0..min(y0+TY, ny),
  // the non-real test over faces -1..ny+1, for updated columns only;
  // first-order faces: r = 0 and r = dx of the axisymmetric form
  const int klo = HALO_Y, khi = min(TY + HALO_Y, D.ny - y0 + HALO_Y);
  const int nlo = max(1, 2 - y0), nhi = D.ny + 4 - y0;
  int glo = 1, ghi = 0;
  if (axi && D.y0 == 0.0 && y0 == 0) { glo = HALO_Y; ghi = HALO_Y + AXIS_FACES - 1; }
  March<LIM, COMP, SPEC> m;
  m.init((float)A.beta, S->lam32);
  YSrc src;
  src.qp0 = src.qp1 = src.qp2 = vs(0.f);
  src.zp2 = src.zp3 = src.zpp2 = src.zpp3 = vs(0.f);
  Cell out;
  for (int c = 0; c < nch; c++) {
    unsigned s = (base + c) % Y32_STAGES;
    unsigned par = ((base + c) / Y32_STAGES) & 1u;
    if (!__all_sync(0xffffffffu, mbar_wait(&bars[s], par, A.wait_polls))) {
      wait_failed(S, &bars[s], par, lane);
      // the remaining chunks of this tile that were issued still land
      for (int d = c + 1; d < nch && d < c + Y32_STAGES; d++) {
        unsigned s2 = (base + d) % Y32_STAGES;
        mbar_wait(&bars[s2], ((base + d) / Y32_STAGES) & 1u);
      }
      return 1;
    }
    const unsigned char *st = ring + s * Y32_STAGE_BYTES;
    const int rows = min(YRB, nrows - c * YRB);
    auto fetch = [&](int i, int j) {
      const int gy = y0 - HALO_Y + j;
      const unsigned char *rp = st + i * (YBOX * 4) + (2 + 2 * lane) * 4;
      float2 f0 = *(const float2 *)(rp);
      float2 f1 = *(const float2 *)(rp + YRB * YBOX * 4);
      float2 f2 = *(const float2 *)(rp + 2 * YRB * YBOX * 4);
      float v[3];
      ycell(D, ca, gy, qi, f0.x, f1.x, f2.x, v);
      f0.x = v[0]; f1.x = v[1]; f2.x = v[2];
      ycell(D, cb, gy, qi, f0.y, f1.y, f2.y, v);
      f0.y = v[0]; f1.y = v[1]; f2.y = v[2];
      // march order of the x2 sweep: (q1 - 1, q3, q2)
      Cell q;
      q.a = f0; q.b = f2; q.c = f1;
      return q;
    };
    // a chunk without border work: its rows and the lanes' columns all
    // inside the domain (no ghost, no override, every row stored by lanes
    // 1..30)
    const int r0 = y0 - HALO_Y + c * YRB;
    const bool plain_chunk = ysweep && rows == YRB && x0 >= 2 && x0 + YW + 2 <= D.nx &&
                             r0 >= 0 && r0 + YRB <= D.ny && r0 - 2 > 0;
    // rows [0, g_end) take the start of the march (first chunk) or the
    // general path (border rules), the rest the plain loop; in a plain
    // chunk the start-up rows are domain cells read as they are, and every
    // face they make is a domain face, so no border rule or accounting mask
    // applies to them either
    const int g_end = plain_chunk ? (c == 0 ? 4 : 0) : rows;
    if (plain_chunk) {
      for (int i = 0; i < g_end; i++) {
        const int j = c * YRB + i;
        const unsigned char *rp = st + i * (YBOX * 4) + (2 + 2 * lane) * 4;
        Cell q;
        q.a = *(const float2 *)(rp);
        q.c = *(const float2 *)(rp + YRB * YBOX * 4);
        q.b = *(const float2 *)(rp + 2 * YRB * YBOX * 4);
        if (m.template push<false>(j, q, out, true, true, true, true, false))
          ysink<false>(src, A, D, x0, y0, TY, lane, y0 - HALO_Y + j - 2, out.a, out.c, out.b,
                       source, axi, coef, dt32, ca, cb, qo);
      }
    }
    for (int i = plain_chunk ? g_end : 0; i < g_end; i++) {
      const int j = c * YRB + i;
      Cell q = fetch(i, j);
      if (!ysweep) {
        if (j >= 2 && j <= nrows - 3)
          ysink<true>(src, A, D, x0, y0, TY, lane, y0 - HALO_Y + j, q.a, q.c, q.b, source, axi,
                      coef, dt32, ca, cb, qo);
        continue;
      }
      bool kin = j >= klo && j <= khi, nin = j >= nlo && j <= nhi;
      bool got = m.template push<true>(j, q, out, kin && ca.upd, kin && cb.upd, nin && ca.upd,
                                       nin && cb.upd, j - 1 >= glo && j - 1 <= ghi);
      if (got)
        ysink<true>(src, A, D, x0, y0, TY, lane, y0 - HALO_Y + j - 2, out.a, out.c, out.b, source,
                    axi, coef, dt32, ca, cb, qo);
    }
    if (plain_chunk) {
      // several rows at a time, so the compiler can overlap consecutive rows
      FVNA_UNROLL(FVNA_Y_UNROLL)
      for (int i = g_end; i < YRB; i++) {
        const int j = c * YRB + i;
        const unsigned char *rp = st + i * (YBOX * 4) + (2 + 2 * lane) * 4;
        Cell q;
        q.a = *(const float2 *)(rp);
        q.c = *(const float2 *)(rp + YRB * YBOX * 4);
        q.b = *(const float2 *)(rp + 2 * YRB * YBOX * 4);
        Cell o = m.template step<false>(q, true, true, true, true, false);
        ysink<false>(src, A, D, x0, y0, TY, lane, y0 - HALO_Y + j - 2, o.a, o.c, o.b, source, axi,
                     coef, dt32, ca, cb, qo);
      }
    }
    // every lane's shared-memory reads of this stage are ordered before its
    // next TMA fill
    fence_async();
    __syncwarp();
    if (lane == 0 && c + Y32_STAGES < nch) issue(c + Y32_STAGES);
  }
  if (SPEC && ysweep && !spec_held(m.acc)) return 2;
  if (ysweep) flush_acc(m.acc, S, lane);
  return 0;
}

}  // namespace x2

// The end of the step in the x2 sweep's second kernel: the last block to
// finish runs the per-domain step end (fvna_step.cuh) once every tile's
// statistics are in.
__device__ __forceinline__ void y32_finish_step(const StepArgs &A, int lane, bool wrote) {
  if (!A.fold_advance) return;
  unsigned prev = 0;
  if (lane == 0) {
    if (wrote) __threadfence();   // this block's statistics before its arrival
    prev = atomicAdd(&A.counters[2], 1u);
  }
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != gridDim.x - 1) return;
  __threadfence();
  for (int d = lane; d < A.ndom; d += 32) advance_domain(A, d);
  if (lane == 0) A.counters[2] = 0u;
}

template <int LIM, bool COMP, bool REDO>
__global__ void __launch_bounds__(32, Y32_MINBLOCKS) k_sweep_y32(StepArgs A) {
  using namespace x2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *ring = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t *bars = (uint64_t *)(ring + Y32_STAGES * Y32_STAGE_BYTES);
  const int lane = threadIdx.x;
  const Maps *maps = (const Maps *)A.tmaps;
  griddep_wait();
  const int nredo = REDO ? A.redo[1] : 0;
  if (REDO && nredo == 0) {
    // nothing to redo: every statistic of the step is in (the first kernel
    // has completed), so block 0 alone ends the step, without arrivals
    if (blockIdx.x == 0) {
      if (lane == 0) A.redo[0] = 0;
      if (A.fold_advance)
        for (int d = lane; d < A.ndom; d += 32) advance_domain(A, d);
    }
    return;
  }
  if (lane == 0)
    for (int s = 0; s < Y32_STAGES; s++) mbar_init(&bars[s], 1);
  if (blockIdx.x == 0 && lane == 0) {
    if (REDO) A.redo[0] = 0;      // the x1 sweep's list, empty for the next step
    else A.counters[0] = 0u;      // the x1 sweep's tile counter
  }
  __syncwarp();
  unsigned used = 0;
  const int nt = REDO ? nredo : A.ntiles;
  int it = REDO ? (int)blockIdx.x : take_tile(&A.counters[1], lane);
  while (it < nt) {
    const unsigned tn = REDO ? 0u : take_tile_issue(&A.counters[1], lane);
    const int w = REDO ? A.redo[A.redo_off + it] : it;
    const int cur = it;
    const Tile tl = A.tiles[w];
    const DomDev &D = A.doms[tl.dom];
    DomScal *S = A.scal + tl.dom;
    if (S->done) {
      it = REDO ? cur + (int)gridDim.x : take_tile_collect(tn);
      continue;
    }
    const int x0 = tl.x0, y0 = tl.y0;
    // one code path for all tiles (border rules are per-row branches that
    // chunks away from the domain edges skip)
    // a tile's height: its own (the host may mix heights), else the sweep's
    const int TY = tl.pad > 0 ? tl.pad : A.tile_y;
    int rc = REDO ? x2::y32_tile<LIM, COMP, false>(A, D, S, maps[tl.dom], ring, bars, used, x0,
                                                    y0, TY, lane)
                  : x2::y32_tile<LIM, COMP, true>(A, D, S, maps[tl.dom], ring, bars, used, x0, y0,
                                                   TY, lane);
    if (rc == 2 && lane == 0) A.redo[A.redo_off + atomicAdd(&A.redo[1], 1)] = w;
    if (rc == 1) break;
    it = REDO ? cur + (int)gridDim.x : take_tile_collect(tn);
  }
  griddep_launch();
  if (REDO) y32_finish_step(A, lane, true);
}

// Analytic border values of the current step into the ghost ring (binary64
// evaluation, eqs. OurTaylorS and hifuBC, rounded once to binary32).
#if FVNA_CHECK
// host reader of the self-check word of this unit (0: no bad index)
static unsigned long long check_word_host() {
  unsigned long long w = 0;
  cudaMemcpyFromSymbol(&w, x2::g_check_word, sizeof w);
  return w;
}
#endif

static __global__ void k_ghost32(StepArgs A, int dom, int always) {
  const DomDev &D = A.doms[dom];
  const DomScal *S = A.scal + dom;
  if ((S->done && !always) || !D.ghost32) return;
  const int nx = D.nx, ny = D.ny;
  const size_t nxr = 6 * (size_t)(ny + 6), n = x2::ghost_ring_size(nx, ny);
  float *R = (float *)D.ghost32;
  const double t = S->t, dx = A.dx;
  const float nan = __int_as_float(0x7fc00000);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v[3];
    bool drv = false;
    if (e < nxr) {
      int k = (int)(e / (ny + 6)), gy = (int)(e - (size_t)k * (ny + 6)) - 3;
      int gx = k < 3 ? k - 3 : nx + k - 3;
      int side = k < 3 ? 0 : 1, bc = D.bc[side];
      double xc = D.x0 + (gx + 0.5) * dx, yc = D.y0 + (gy + 0.5) * dx;
      if (bc == BC_TAYLOR) { P32::taylor(D, xc, yc, t, v); drv = true; }
      else if (bc == BC_HIFU && side == 0 && yc >= 0.0 && yc <= D.aperture) {
        P32::hifu(D, xc, yc, t, v);
        drv = true;
      }
    } else {
      size_t f = e - nxr;
      int k = (int)(f / (nx + 6)), cx = (int)(f - (size_t)k * (nx + 6)) - 3;
      int gy = k < 3 ? k - 3 : ny + k - 3;
      int bc = D.bc[k < 3 ? 2 : 3];
      if (bc == BC_TAYLOR) {
        P32::taylor(D, D.x0 + (cx + 0.5) * dx, D.y0 + (gy + 0.5) * dx, t, v);
        drv = true;
      }
    }
    R[e] = drv ? (float)v[0] : nan;
    R[n + e] = drv ? (float)v[1] : nan;
    R[2 * n + e] = drv ? (float)v[2] : nan;
  }
}

}  // namespace fvna
