// fvna_xh.cuh -- the binary32 x1 sweep with the lanes along x1 (arXiv
// 1311.3004, section 3: Roe solver, MC-limited corrections and the update of
// eq. fv-hr along x1, in the perturbation variables).
//
// A warp takes one segment at a time: two adjacent rows (one packed FP32x2
// pair, .x the first row, .y the second) and 64 consecutive cells, lane l
// holding cells x0 - 2 + 2l and x0 - 1 + 2l.  Each lane computes the two
// faces on the left of its cells; the neighbour faces the limiter ratio
// needs, the left neighbour cell and the fluctuation of the next face come
// from the adjacent lanes by shuffles.  Lanes 1..30 update and store their
// cells: 60 cells per row and segment, the first and last two being the
// halo.  Loads and stores are coalesced 8-byte accesses, nothing is staged
// in shared memory, and no state is carried from one segment to the next.
//
// As in the other binary32 sweeps every face is first taken as subsonic; a
// segment that met another face (or a sound-speed deviation outside the
// series range) is recomputed with the general split.
#pragma once

#include "fvna_sweeps32.cuh"

namespace fvna {

constexpr int XH_OUT = 60;      // cells a segment updates per row (64 marched)
constexpr int XH_TILE = 60;     // fvna_config.tile_x value that selects this kernel
#ifndef XH_MINBLOCKS
#define XH_MINBLOCKS 14   // the compiler settles at 128 registers, no spills: 16 warps per SM
#endif

namespace x2 {

__device__ __forceinline__ V shup(V a) {
  return make_float2(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1));
}
__device__ __forceinline__ V shdn(V a) {
  return make_float2(__shfl_down_sync(0xffffffffu, a.x, 1),
                     __shfl_down_sync(0xffffffffu, a.y, 1));
}

// merge the statistics of a segment into the running ones of the warp
__device__ __forceinline__ void acc_merge(Acc &t, const Acc &a) {
  t.smax.x = max3_abs_nan(t.smax.x, a.smax.x, 0.f);
  t.smax.y = max3_abs_nan(t.smax.y, a.smax.y, 0.f);
  t.c2min.x = fminf(t.c2min.x, a.c2min.x);
  t.c2min.y = fminf(t.c2min.y, a.c2min.y);
}
__device__ __forceinline__ void acc_init(Acc &a) {
  a.smax = vs(0.f);
  a.c2min = vs(1.f);
  a.sub = vs(1.f);
  a.dmax = vs(0.f);
}

// value of cell (gx, gy) of a border segment: the state for cells inside the
// domain, the border rules of load32 for the rest
__device__ __forceinline__ void xh_cell(const DomDev &D, const float *const q[3], int gx, int gy,
                                        float v[3]) {
  if (gx >= 0 && gx < D.nx) {
    size_t o = (size_t)gy * D.pitch + gx;
    v[0] = q[0][o]; v[1] = q[1][o]; v[2] = q[2][o];
    return;
  }
  load32(D, q, gx, gy, v);
}

// The cells of an interior segment (both rows inside, cells x0 - 2 ..
// x0 + 61 inside the domain): three coalesced 8-byte loads per row.
__device__ __forceinline__ void xh_load(const DomDev &D, int x0, int y0, int lane, Cell &Ca,
                                        Cell &Cb) {
  const size_t o0 = (size_t)y0 * D.pitch + (x0 - 2 + 2 * lane);
  const size_t o1 = o0 + (size_t)D.pitch;
  float2 r0[3], r1[3];
#pragma unroll
  for (int f = 0; f < 3; f++) {
    r0[f] = __ldg((const float2 *)((const float *)D.qa[f] + o0));
    r1[f] = __ldg((const float2 *)((const float *)D.qa[f] + o1));
  }
  Ca.a = make_float2(r0[0].x, r1[0].x); Cb.a = make_float2(r0[0].y, r1[0].y);
  Ca.b = make_float2(r0[1].x, r1[1].x); Cb.b = make_float2(r0[1].y, r1[1].y);
  Ca.c = make_float2(r0[2].x, r1[2].x); Cb.c = make_float2(r0[2].y, r1[2].y);
}
__device__ __forceinline__ bool xh_interior(const DomDev &D, int x0, int y0) {
  return x0 >= 2 && x0 + XH_OUT + 2 <= D.nx && y0 + 2 <= D.ny;
}

// One segment; an interior one (BORDER off) takes its cells from Ca, Cb
// (loaded by xh_load), a border one loads them itself with the border rules.
// Returns false (statistics untouched) when SPEC met a face that is not
// subsonic; the caller then recomputes it with SPEC off.
template <int LIM, bool COMP, bool BORDER, bool SPEC>
__device__ __forceinline__ bool xh_segment(const StepArgs &A, const DomDev &D, DomScal *S, int x0,
                                           int y0, int lane, Cell Ca, Cell Cb, Acc &tot) {
  const int nx = D.nx, ny = D.ny;
  const int ca = x0 - 2 + 2 * lane;
  const bool row1 = y0 + 1 < ny;
  float *qo[3] = {(float *)D.qb[0], (float *)D.qb[1], (float *)D.qb[2]};
  const size_t o0 = (size_t)y0 * D.pitch + ca;
  const size_t o1 = o0 + (size_t)D.pitch;
  if (BORDER) {
    const float *q[3] = {(const float *)D.qa[0], (const float *)D.qa[1],
                         (const float *)D.qa[2]};
    const int gy1 = row1 ? y0 + 1 : y0;
    float v[3];
    xh_cell(D, q, ca, y0, v);      Ca.a.x = v[0]; Ca.b.x = v[1]; Ca.c.x = v[2];
    xh_cell(D, q, ca, gy1, v);     Ca.a.y = v[0]; Ca.b.y = v[1]; Ca.c.y = v[2];
    xh_cell(D, q, ca + 1, y0, v);  Cb.a.x = v[0]; Cb.b.x = v[1]; Cb.c.x = v[2];
    xh_cell(D, q, ca + 1, gy1, v); Cb.a.y = v[0]; Cb.b.y = v[1]; Cb.c.y = v[2];
  }
  const V bm1 = vs((float)A.beta - 1.f);
  const float lam = A.x_half ? 0.5f * S->lam32 : S->lam32;   // dt/dx (halved: Strang)
  const V nhlam = vs(-0.5f * lam), nlam = vs(-lam);
  V zbA, zcA, zbB, zcB;
  zof(Ca, zbA, zcA);
  zof(Cb, zbB, zcB);
  // the left neighbour of cell ca is the previous lane's second cell
  Cell Cl;
  Cl.a = shup(Cb.a); Cl.b = shup(Cb.b); Cl.c = shup(Cb.c);
  const V zbl = shup(zbB), zcl = shup(zcB);
  Face FA, FB;
  V dmA, dmB;
  const V c2A = roe<SPEC>(bm1, Cl, zbl, zcl, Ca, zbA, zcA, FA, dmA);
  const V c2B = roe<SPEC>(bm1, Ca, zbA, zcA, Cb, zbB, zcB, FB, dmB);
  // statistics: face A of lane 0 has no left cell; in border segments |s|
  // counts over the domain's faces and the non-real test over the extended
  // line's, as in the tile sweeps
  Acc acc;
  acc_init(acc);
  if (!BORDER) {
    if (lane > 0) {
      acc_face(acc, FA, c2A);
      if (SPEC) acc_dm(acc, dmA);
    }
    acc_face(acc, FB, c2B);
    if (SPEC) acc_dm(acc, dmB);
  } else {
    auto mask = [&](int gl, bool &sx, bool &sy, bool &nx_, bool &ny_) {
      sx = gl >= -1 && gl <= nx - 1;
      nx_ = gl >= -2 && gl <= nx;
      sy = sx && row1;
      ny_ = nx_ && row1;
    };
    bool sx, sy, nx_, ny_;
    if (lane > 0) {
      mask(ca - 1, sx, sy, nx_, ny_);
      acc_face_masked(acc, FA, c2A, sx, sy, nx_, ny_);
      if (SPEC) acc_dm(acc, dmA);
    }
    mask(ca, sx, sy, nx_, ny_);
    acc_face_masked(acc, FB, c2B, sx, sy, nx_, ny_);
    if (SPEC) acc_dm(acc, dmB);
  }
  if (SPEC && !spec_held(acc)) return false;
  // neighbour faces: the previous lane's face B (left of A), the next lane's
  // face A (right of B); the subsonic split reads only the upwind families
  Face LB, RA;
  LB.a1 = shup(FB.a1); LB.s0 = shup(FB.s0); LB.r13 = shup(FB.r13); LB.a3 = shup(FB.a3);
  RA.a2 = shdn(FA.a2); RA.s1 = shdn(FA.s1); RA.r23 = shdn(FA.r23); RA.a3 = shdn(FA.a3);
  if (!SPEC) {
    LB.a2 = shup(FB.a2); LB.s1 = shup(FB.s1); LB.r23 = shup(FB.r23);
    RA.a1 = shdn(FA.a1); RA.s0 = shdn(FA.s0); RA.r13 = shdn(FA.r13);
  }
  V PA[3], MA[3], PB[3], MB[3];
  flux<LIM, SPEC>(FA, LB, FB, nhlam, false, PA, MA);
  flux<LIM, SPEC>(FB, FA, RA, nhlam, false, PB, MB);
  // the right face of cell ca + 1 is the next lane's face A
  V MAn[3] = {shdn(MA[0]), shdn(MA[1]), shdn(MA[2])};
  Cell Na, Nb;
  Na.a = update<COMP>(Ca.a, PA[0], MB[0], nlam);
  Na.b = update<COMP>(Ca.b, PA[1], MB[1], nlam);
  Na.c = update<COMP>(Ca.c, PA[2], MB[2], nlam);
  Nb.a = update<COMP>(Cb.a, PB[0], MAn[0], nlam);
  Nb.b = update<COMP>(Cb.b, PB[1], MAn[1], nlam);
  Nb.c = update<COMP>(Cb.c, PB[2], MAn[2], nlam);
  if (lane >= 1 && lane <= 30) {
    if (!BORDER) {
      *(float2 *)(qo[0] + o0) = make_float2(Na.a.x, Nb.a.x);
      *(float2 *)(qo[1] + o0) = make_float2(Na.b.x, Nb.b.x);
      *(float2 *)(qo[2] + o0) = make_float2(Na.c.x, Nb.c.x);
      *(float2 *)(qo[0] + o1) = make_float2(Na.a.y, Nb.a.y);
      *(float2 *)(qo[1] + o1) = make_float2(Na.b.y, Nb.b.y);
      *(float2 *)(qo[2] + o1) = make_float2(Na.c.y, Nb.c.y);
    } else {
      if (ca < nx) {
        qo[0][o0] = Na.a.x; qo[1][o0] = Na.b.x; qo[2][o0] = Na.c.x;
        if (row1) { qo[0][o1] = Na.a.y; qo[1][o1] = Na.b.y; qo[2][o1] = Na.c.y; }
      }
      if (ca + 1 < nx) {
        qo[0][o0 + 1] = Nb.a.x; qo[1][o0 + 1] = Nb.b.x; qo[2][o0 + 1] = Nb.c.x;
        if (row1) { qo[0][o1 + 1] = Nb.a.y; qo[1][o1 + 1] = Nb.b.y; qo[2][o1 + 1] = Nb.c.y; }
      }
    }
  }
  acc_merge(tot, acc);
  return true;
}

}  // namespace x2

// The x1 sweep: warps take segments (two rows x 60 updated cells) from the
// sweep's counter, segments at a domain border first; statistics are
// gathered per warp and flushed when the domain changes and at the end.
template <int LIM, bool COMP>
__global__ void __launch_bounds__(32, XH_MINBLOCKS) k_sweep_x32h(StepArgs A) {
  using namespace x2;
  const int lane = threadIdx.x;
  griddep_wait();
  if (blockIdx.x == 0 && lane == 0) {
    A.counters[1] = 0u;         // the x2 sweep's tile counter
    A.redo[1] = 0;              // the x2 sweep's list, empty for this step
  }
  if (!(A.sweeps & 1)) {
    // x1 sweep off: the swept planes take the state as it is
    for (int d = 0; d < A.ndom; d++) {
      if (A.scal[d].done) continue;
      const DomDev &D = A.doms[d];
      const size_t n = (size_t)D.ny * D.pitch;
      for (int f = 0; f < 3; f++)
        for (size_t i = (size_t)blockIdx.x * 32 + lane; i < n; i += (size_t)gridDim.x * 32)
          ((float *)D.qb[f])[i] = ((const float *)D.qa[f])[i];
    }
    return;
  }
  const int nt = A.ntiles;
  Acc tot;
  acc_init(tot);
  int cur = -1;
  int it = take_tile(&A.counters[0], lane);
  while (it < nt) {
    // the next segment is claimed when this one starts and collected when it ends
    const unsigned tn = take_tile_issue(&A.counters[0], lane);
    const Tile tl = A.tiles[it];
    if (tl.dom != cur) {
      if (cur >= 0) flush_acc(tot, A.scal + cur, lane);
      acc_init(tot);
      cur = tl.dom;
    }
    const DomDev &D = A.doms[tl.dom];
    DomScal *S = A.scal + tl.dom;
    if (!S->done) {
      const int x0 = tl.x0, y0 = tl.y0;
      Cell Ca, Cb;
      bool ok;
      if (xh_interior(D, x0, y0)) {
        xh_load(D, x0, y0, lane, Ca, Cb);
        ok = xh_segment<LIM, COMP, false, true>(A, D, S, x0, y0, lane, Ca, Cb, tot);
      } else {
        ok = xh_segment<LIM, COMP, true, true>(A, D, S, x0, y0, lane, Ca, Cb, tot);
      }
      if (!ok) xh_segment<LIM, COMP, true, false>(A, D, S, x0, y0, lane, Ca, Cb, tot);
    }
    it = take_tile_collect(tn);
  }
  griddep_launch();
  if (cur >= 0) flush_acc(tot, A.scal + cur, lane);
}

}  // namespace fvna
