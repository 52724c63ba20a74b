// fvna_x2.cuh -- building blocks of the binary32 sweeps: packed two-lane
// arithmetic, TMA / mbarrier wrappers, and the line march on pairs of
// independent lines (arXiv 1311.3004, section 3: Roe solver, MC-limited
// corrections, update of eq. fv-hr), in the perturbation variables
// (q1 - 1, q2, q3).
//
// Every lane marches two independent lines at once; a pair value holds the
// two lines' numbers and most arithmetic runs as one packed FP32x2
// instruction (add/mul/fma .f32x2).  Divisions and square roots use the
// hardware approximations (one MUFU each, relative error below 2^-22);
// min/max, compares and selects stay per line.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fvna_types.h"

namespace fvna {
namespace x2 {

typedef float2 V;

__device__ __forceinline__ V vs(float a) { return make_float2(a, a); }
__device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
// a - b, exact as one rounding (b * -1 is exact)
__device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// c - a * b
__device__ __forceinline__ V fnma(V a, V b, V c) {
  return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}

__device__ __forceinline__ float rcp1(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt1(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ V rcp(V a) { return make_float2(rcp1(a.x), rcp1(a.y)); }
__device__ __forceinline__ V rsqrt(V a) { return make_float2(rsqrt1(a.x), rsqrt1(a.y)); }

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
// max(|a|, |b|, |c|), NaN if any input is NaN
__device__ __forceinline__ float max3_abs_nan(float a, float b, float c) {
  float r;
  asm("max.NaN.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// ---------------------------------------------------------------------------
// TMA and mbarrier (PTX: cp.async.bulk.tensor, mbarrier.*)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned su32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a phase of `bar`: at most `limit` polls.  Every try_wait
// may suspend the thread for a while, so the default limit is a few seconds
// at most; false means the copy did not arrive in time (the caller records
// an error, waits once more with the default limit for the copy to land, and
// stops using the buffer).
constexpr int WAIT_LIMIT = 1 << 22;

// Programmatic dependent launch of the binary32 sweeps: griddep_wait blocks
// until the grid this one follows in the stream has completed and its
// memory is visible (at once in a launch without the attribute, or when
// that grid has already completed); griddep_launch lets the next grid start
// launching once every block of this one has called it or exited.  Each
// sweep kernel waits before its first global access and signals when its
// block takes no more tiles.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          int limit = WAIT_LIMIT) {
  for (int i = 0; i < limit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(su32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::
                   "l"(map),
               "r"(x), "r"(y), "r"(su32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses
__device__ __forceinline__ void fence_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Tensor maps of one domain for the binary32 sweeps (built on the host).
struct Maps {
  CUtensorMap xin[3];    // state planes, box SW x 32, swizzled (x1 sweep loads)
  CUtensorMap xhalo[3];  // state planes, box 4 x 32 (x1 sweep halo columns)
  CUtensorMap xout[3];   // swept planes, box SW x 32, swizzled (x1 sweep stores)
  CUtensorMap yin[3];    // swept planes, box YBOX x YRB (x2 sweep loads)
};
// x2 sweep: a warp marches 64 columns (two per lane) starting 2 left of its
// tile and updates the 60 in the middle; its loads cover 68 columns from 4
// left of the tile (16-byte aligned start) in chunks of YRB rows.
constexpr int YW = 60;
constexpr int YBOX = 68;
constexpr int YRB = 8;

// ---------------------------------------------------------------------------
// One interface of a pair of lines (Roe solver of section 3.2 on the
// perturbation variables).
// ---------------------------------------------------------------------------
struct Face {
  V s0, s1, u, r13, r23, a1, a2, a3;
};
struct Cell {
  V a, b, c;
};

// z = (q2, q3) / q1 of a cell, q1 = 1 + a
__device__ __forceinline__ void zof(const Cell &q, V &zb, V &zc) {
  V r = rcp(add(q.a, vs(1.f)));
  zb = mul(q.b, r);
  zc = mul(q.c, r);
}

// Roe average, speeds and waves between L and R.  bm1 = beta - 1.  Returns
// c^2 = 1 + (D - 1) (negative: non-real speeds) and D - 1 in dm.  SERIES:
// 1/c from its Taylor series in D - 1 (valid for |D - 1| < DM_SERIES, where
// its truncation error is below 2e-10; the march records max |D - 1| and a
// tile beyond that range is redone without SERIES).
constexpr float DM_SERIES = 0.03f;
template <bool SERIES>
__device__ __forceinline__ V roe(V bm1, const Cell &L, V zbL, V zcL, const Cell &R, V zbR, V zcR,
                                 Face &F, V &dm_out) {
  V S1 = add(L.a, R.a);           // 2 (Z1 - 1)
  V S2 = add(zbL, zbR);           // 2 Z2
  V S3 = add(zcL, zcR);           // 2 Z3
  V rz = rcp(add(S1, vs(2.f)));   // 1 / (2 Z1)
  V u = mul(S2, rz);
  V v = mul(S3, rz);
  V tt = sub(u, S2);              // u - 2 Z2
  V dm = fma(u, tt, mul(bm1, S1));  // D - 1 = u^2 - 2 Z2 u + beta2 (Z1 - 1)
  V c2 = add(dm, vs(1.f));
  dm_out = dm;
  V c, rc;
  if (SERIES) {
    // 1/sqrt(1 + dm) = 1 - dm/2 + 3dm^2/8 - 5dm^3/16 + 35dm^4/128 - 63dm^5/256
    rc = fma(dm, vs(-63.f / 256.f), vs(35.f / 128.f));
    rc = fma(dm, rc, vs(-5.f / 16.f));
    rc = fma(dm, rc, vs(3.f / 8.f));
    rc = fma(dm, rc, vs(-0.5f));
    rc = fma(dm, rc, vs(1.f));
    c = fma(dm, rc, rc);   // (1 + dm) / sqrt(1 + dm), without rounding 1 + dm first
  } else {
    // c - 1 = dm / (1 + sqrt(1 + dm)) keeps the relative precision of dm, so
    // c = 1 + (c - 1) is rounded once, and 1/c gets one Newton step: both set
    // the propagation speed of every wave, where an error of the hardware
    // approximations (~1e-7, one-signed) would add up step after step
    c = add(mul(dm, rcp(fma(c2, rsqrt(c2), vs(1.f)))), vs(1.f));
    rc = rcp(c);
    rc = fma(rc, fma(make_float2(-c.x, -c.y), rc, vs(1.f)), rc);
  }
  V nc1 = sub(c, u);
  F.u = u;
  F.s0 = add(u, c);
  F.s1 = sub(u, c);
  V d1 = sub(R.a, L.a), d2 = sub(R.b, L.b), d3 = sub(R.c, L.c);
  V h = mul(rc, vs(0.5f));
  F.a1 = mul(fma(nc1, d1, d2), h);          // (d2 - s1 d1) / (2c)
  F.a2 = mul(sub(mul(F.s0, d1), d2), h);    // (s0 d1 - d2) / (2c)
  V w = mul(v, rc);
  F.r13 = mul(w, add(tt, c));               // v (s0 - 2 Z2) / c
  F.r23 = mul(w, sub(c, tt));               // v (2 Z2 - s1) / c
  F.a3 = sub(d3, fma(F.a1, F.r13, mul(F.a2, F.r23)));
  return c2;
}

// Limiter of eq. limiter for theta = num / den, on both lines: MC
// max(0, min(2 theta, (1 + theta) / 2, 2)); none: 0; Lax-Wendroff: 1.  A
// zero wave (den = 0) may give any finite value: its correction is phi * 0.
template <int LIM> __device__ __forceinline__ V phi(V num, V den) {
  if (LIM == LIM_NONE) return vs(0.f);
  if (LIM == LIM_LW) return vs(1.f);
  V th = mul(num, rcp(den));
  V t2 = add(th, th);
  V th1 = fma(th, vs(0.5f), vs(0.5f));
  return make_float2(fmaxf(min3(t2.x, th1.x, 2.f), 0.f), fmaxf(min3(t2.y, th1.y, 2.f), 0.f));
}

__device__ __forceinline__ V vmax0(V a) { return make_float2(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f)); }
__device__ __forceinline__ V vmin0(V a) { return make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f)); }
__device__ __forceinline__ V vabs(V a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
// per line: s > 0 ? l : r
__device__ __forceinline__ V upwind(V s, V l, V r) {
  return make_float2(s.x > 0.f ? l.x : r.x, s.y > 0.f ? l.y : r.y);
}

// A face that is not subsonic on both lines (never met by acoustic
// perturbations): each family on its own side, per line.
struct PM {
  V P0, P1, P2, M0, M1, M2;
};
template <int LIM>
__device__ __forceinline__ PM flux_general(const Face I, const Face Lf, const Face Rf, V nhlam,
                                        bool first_order, V g2, V up, V um) {
  V U0a = upwind(I.s0, Lf.a1, Rf.a1), U0s = upwind(I.s0, Lf.s0, Rf.s0);
  V U0r = upwind(I.s0, Lf.r13, Rf.r13);
  V U1a = upwind(I.s1, Lf.a2, Rf.a2), U1s = upwind(I.s1, Lf.s1, Rf.s1);
  V U1r = upwind(I.s1, Lf.r23, Rf.r23);
  V N0 = fma(I.r13, I.r13, fma(I.s0, I.s0, vs(1.f)));
  V D0 = fma(U0r, I.r13, fma(U0s, I.s0, vs(1.f)));
  V N1 = fma(I.r23, I.r23, fma(I.s1, I.s1, vs(1.f)));
  V D1 = fma(U1r, I.r23, fma(U1s, I.s1, vs(1.f)));
  V as0 = vabs(I.s0), as1 = vabs(I.s1);
  V g0 = mul(mul(mul(as0, fma(nhlam, as0, vs(0.5f))), phi<LIM>(mul(U0a, D0), mul(I.a1, N0))), I.a1);
  V g1 = mul(mul(mul(as1, fma(nhlam, as1, vs(0.5f))), phi<LIM>(mul(U1a, D1), mul(I.a2, N1))), I.a2);
  if (first_order) g0 = g1 = g2 = vs(0.f);
  V F0 = add(g0, g1);
  V F1 = fma(g1, I.s1, mul(g0, I.s0));
  V F2 = fma(g0, I.r13, fma(g1, I.r23, g2));
  V s0p = vmax0(I.s0), s0m = vmin0(I.s0), s1p = vmax0(I.s1), s1m = vmin0(I.s1);
  V w01 = mul(I.a1, I.s0), w02 = mul(I.a1, I.r13);
  V w11 = mul(I.a2, I.s1), w12 = mul(I.a2, I.r23);
  PM r;
  r.P0 = sub(fma(s1p, I.a2, mul(s0p, I.a1)), F0);
  r.P1 = sub(fma(s1p, w11, mul(s0p, w01)), F1);
  r.P2 = sub(fma(up, I.a3, fma(s1p, w12, mul(s0p, w02))), F2);
  r.M0 = add(fma(s1m, I.a2, mul(s0m, I.a1)), F0);
  r.M1 = add(fma(s1m, w11, mul(s0m, w01)), F1);
  r.M2 = add(fma(um, I.a3, fma(s1m, w12, mul(s0m, w02))), F2);
  return r;
}

// Fluctuations (eqs. fluc:m, fluc:p) and the limited correction flux (eq.
// limiter) of face I, folded into P = A+dq - F (what the face adds to the
// cell on its right) and M = A-dq + F (to the cell on its left), so that the
// update of eq. fv-hr reads q -= lam (P_left + M_right).  Lf / Rf are the
// neighbour faces for the upwind ratio; nhlam = -lam / 2; first_order drops
// the correction (F = 0).
//
// With W0 = a1 (1, s0, r13), W1 = a2 (1, s1, r23), W2 = (0, 0, a3) the
// limiter ratio of family p is (U_p . W_p) / (W_p . W_p) = a_up D / (a N)
// with N = r.r and D = r_up . r, and (1/2) |s| (1 - lam |s|) phi W_p =
// g_p (1, s, r) with g_p = (1/2 - lam |s| / 2) phi |s| a_p.
template <int LIM, bool SPEC>
__device__ __forceinline__ void flux(const Face &I, const Face &Lf, const Face &Rf, V nhlam,
                                     bool first_order, V P[3], V M[3]) {
  const V up = vmax0(I.u), um = vmin0(I.u);
  // family 3 (speed u, transverse momentum only)
  const V au = vabs(I.u);
  V g2 = mul(mul(mul(au, fma(nhlam, au, vs(0.5f))), phi<LIM>(upwind(I.u, Lf.a3, Rf.a3), I.a3)),
             I.a3);
  // SPEC: the face is taken as subsonic (the march records min(s0, -s1) and
  // the caller redoes the tile with SPEC off if some face was not)
  if (SPEC) {
    // subsonic face: family 1 moves right (upwind = left face), family 2
    // left (upwind = right face); A-dq has no family-1 term, A+dq none of
    // family 2
    V N0 = fma(I.r13, I.r13, fma(I.s0, I.s0, vs(1.f)));
    V D0 = fma(Lf.r13, I.r13, fma(Lf.s0, I.s0, vs(1.f)));
    V N1 = fma(I.r23, I.r23, fma(I.s1, I.s1, vs(1.f)));
    V D1 = fma(Rf.r23, I.r23, fma(Rf.s1, I.s1, vs(1.f)));
    V p0 = mul(I.a1, I.s0);   // s0 a1 = |s0| a1
    V q1 = mul(I.a2, I.s1);   // s1 a2 = -|s1| a2
    // g0 and -g1
    V g0 = mul(mul(p0, fma(nhlam, I.s0, vs(0.5f))), phi<LIM>(mul(Lf.a1, D0), mul(I.a1, N0)));
    V ng1 = mul(mul(q1, sub(vs(0.5f), mul(nhlam, I.s1))),
                phi<LIM>(mul(Rf.a2, D1), mul(I.a2, N1)));
    if (first_order) g0 = ng1 = g2 = vs(0.f);
    V F0 = sub(g0, ng1);
    V F1 = sub(mul(g0, I.s0), mul(ng1, I.s1));
    V F2 = sub(fma(g0, I.r13, g2), mul(ng1, I.r23));
    P[0] = sub(p0, F0);
    P[1] = sub(mul(p0, I.s0), F1);
    P[2] = sub(fma(up, I.a3, mul(p0, I.r13)), F2);
    M[0] = add(q1, F0);
    M[1] = fma(q1, I.s1, F1);
    M[2] = fma(q1, I.r23, fma(um, I.a3, F2));
    return;
  }
  PM r = flux_general<LIM>(I, Lf, Rf, nhlam, first_order, g2, up, um);
  P[0] = r.P0; P[1] = r.P1; P[2] = r.P2;
  M[0] = r.M0; M[1] = r.M1; M[2] = r.M2;
}

// Update of eq. fv-hr, q - lam (P_left + M_right), nlam = -lam.  Without
// COMP the two increments are summed first and the state is rounded once
// (one fused multiply-add).  With COMP the state and the two increments are
// summed with error-free two-sums and the rounding errors folded back once
// (Neumaier), so the result is the exact sum of the three, rounded once.
__device__ __forceinline__ void two_sum(V a, V b, V &s, V &e) {
  s = add(a, b);
  V bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
}
template <bool COMP> __device__ __forceinline__ V update(V q, V Pl, V Mr, V nlam) {
  if (!COMP) return fma(nlam, add(Pl, Mr), q);
  V t1 = mul(nlam, Pl), t2 = mul(nlam, Mr);
  V s, e1, e2;
  two_sum(q, t1, s, e1);
  two_sum(s, t2, s, e2);
  return add(s, add(e1, e2));
}

// Running per-line statistics of a march: max |s| (NaN-propagating), the
// smallest c^2 (negative: non-real speeds somewhere) and the smallest
// min(s0, -s1) (not positive: a face that is not subsonic).
struct Acc {
  V smax, c2min, sub, dmax;
};
__device__ __forceinline__ void acc_dm(Acc &A, V dm) {
  A.dmax.x = max3_abs_nan(A.dmax.x, dm.x, 0.f);
  A.dmax.y = max3_abs_nan(A.dmax.y, dm.y, 0.f);
}
__device__ __forceinline__ void acc_face(Acc &A, const Face &F, V c2) {
  A.smax.x = max3_abs_nan(A.smax.x, F.s0.x, F.s1.x);
  A.smax.y = max3_abs_nan(A.smax.y, F.s0.y, F.s1.y);
  A.c2min.x = fminf(A.c2min.x, c2.x);
  A.c2min.y = fminf(A.c2min.y, c2.y);
  A.sub.x = min3(A.sub.x, F.s0.x, -F.s1.x);
  A.sub.y = min3(A.sub.y, F.s0.y, -F.s1.y);
}
__device__ __forceinline__ void acc_face_masked(Acc &A, const Face &F, V c2, bool sx, bool sy,
                                                bool nx_, bool ny_) {
  if (sx) A.smax.x = max3_abs_nan(A.smax.x, F.s0.x, F.s1.x);
  if (sy) A.smax.y = max3_abs_nan(A.smax.y, F.s0.y, F.s1.y);
  if (nx_) A.c2min.x = fminf(A.c2min.x, c2.x);
  if (ny_) A.c2min.y = fminf(A.c2min.y, c2.y);
  A.sub.x = min3(A.sub.x, F.s0.x, -F.s1.x);
  A.sub.y = min3(A.sub.y, F.s0.y, -F.s1.y);
}

// Did a speculative march stay within its assumptions (every face subsonic,
// |D - 1| inside the series range)?  NaN counts as within (it is reported
// through max |s|).
__device__ __forceinline__ bool spec_held(const Acc &A) {
  bool bad = A.sub.x <= 0.f || A.sub.y <= 0.f || A.dmax.x >= DM_SERIES || A.dmax.y >= DM_SERIES;
  return !__any_sync(0xffffffffu, bad);
}

// ---------------------------------------------------------------------------
// The line march on a pair of lines.  Cells j = 0, 1, ... are pushed in
// order; face j lies between cells j-1 and j.  From j = 4 on, every push
// completes the flux of face j-1 and updates cell j-2 (returned through
// `out`, true when an update was produced).
// ---------------------------------------------------------------------------
template <int LIM, bool COMP, bool SPEC> struct March {
  V bm1, nhlam, nlam;
  Cell c1, c2;        // cells j-1 and j-2 (old values)
  V zb1, zc1;         // z of cell j-1
  Face fl, fm;        // faces j-2 and j-1
  V Pl[3];            // P of face j-2 (left face of cell j-2)
  Acc acc;

  __device__ __forceinline__ void init(float beta, float lam) {
    bm1 = vs(beta - 1.f);
    nhlam = vs(-0.5f * lam);
    nlam = vs(-lam);
    acc.smax = vs(0.f);
    acc.c2min = vs(1.f);
    acc.sub = vs(1.f);
    acc.dmax = vs(0.f);
  }
  // MASK: per-face accounting masks (border tiles); fo: first-order face
  template <bool MASK>
  __device__ __forceinline__ bool push(int j, const Cell &q, Cell &out, bool sx, bool sy, bool nx_,
                                       bool ny_, bool fo_prev) {
    V zb, zc;
    zof(q, zb, zc);
    bool done = false;
    if (j == 0) {
      c1 = q; zb1 = zb; zc1 = zc;
      return false;
    }
    Face f;
    V dm;
    V c2v = roe<SPEC>(bm1, c1, zb1, zc1, q, zb, zc, f, dm);
    if (MASK) acc_face_masked(acc, f, c2v, sx, sy, nx_, ny_);
    else acc_face(acc, f, c2v);
    if (SPEC) acc_dm(acc, dm);
    if (j >= 3) {
      // flux of face j-1 (neighbours: faces j-2 and j)
      V P[3], Mr[3];
      flux<LIM, SPEC>(fm, fl, f, nhlam, fo_prev, P, Mr);
      if (j >= 4) {
        out.a = update<COMP>(c2.a, Pl[0], Mr[0], nlam);
        out.b = update<COMP>(c2.b, Pl[1], Mr[1], nlam);
        out.c = update<COMP>(c2.c, Pl[2], Mr[2], nlam);
        done = true;
      }
      Pl[0] = P[0]; Pl[1] = P[1]; Pl[2] = P[2];
    }
    fl = fm;
    fm = f;
    c2 = c1;
    c1 = q; zb1 = zb; zc1 = zc;
    return done;
  }
  // push of a cell j >= 4 (no start-up cases, so consecutive steps can be
  // interleaved by the compiler); returns the update of cell j-2
  template <bool MASK>
  __device__ __forceinline__ Cell step(const Cell &q, bool sx, bool sy, bool nx_, bool ny_,
                                       bool fo_prev) {
    V zb, zc;
    zof(q, zb, zc);
    Face f;
    V dm;
    V c2v = roe<SPEC>(bm1, c1, zb1, zc1, q, zb, zc, f, dm);
    if (MASK) acc_face_masked(acc, f, c2v, sx, sy, nx_, ny_);
    else acc_face(acc, f, c2v);
    if (SPEC) acc_dm(acc, dm);
    V P[3], Mr[3];
    flux<LIM, SPEC>(fm, fl, f, nhlam, fo_prev, P, Mr);
    Cell out;
    out.a = update<COMP>(c2.a, Pl[0], Mr[0], nlam);
    out.b = update<COMP>(c2.b, Pl[1], Mr[1], nlam);
    out.c = update<COMP>(c2.c, Pl[2], Mr[2], nlam);
    Pl[0] = P[0]; Pl[1] = P[1]; Pl[2] = P[2];
    fl = fm;
    fm = f;
    c2 = c1;
    c1 = q; zb1 = zb; zc1 = zc;
    return out;
  }
};

}  // namespace x2
}  // namespace fvna
