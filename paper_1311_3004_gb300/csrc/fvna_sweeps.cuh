// fvna_sweeps.cuh -- the step kernels, templated on the precision policy.
//
//   k_sweep_x  x1 sweep (eq. fv-hr along rows), from the state planes into
//              the second planes.  One warp owns a tile of 32 rows x TX cells; the tile plus a 2-cell halo is copied into
//              shared memory with cp.async (coalesced along rows), then each
//              lane marches one row with the Roe solver and writes the
//              updated cells back in place; the warp stores the tile.
//   k_sweep_y  x2 sweep (entries 2 and 3 switched) fused with the source
//              sub-step.  One warp owns 32 adjacent columns (30 updated,
//              two neighbours for the source's Laplacian) and TY rows; each
//              lane marches its column, rows arrive through a cp.async ring
//              in shared memory (coalesced along the row), and the source is
//              applied one row behind the sweep, with the x neighbours taken
//              from the adjacent lanes by warp shuffles.
// Both keep every interface's waves in registers (computed once per line),
// reduce max|s| with warp shuffles and raise one atomic per warp tile.
#pragma once

#include "fvna_device.cuh"

// Tuning knobs (compile-time): unroll factor of the line march's steady loop
// and the minimum resident blocks per SM requested from the register
// allocator for each sweep.
#ifndef FVNA_MARCH_UNROLL
#define FVNA_MARCH_UNROLL 0   // 0: leave the choice to the compiler
#endif
#ifndef FVNA_X_MINBLOCKS
#define FVNA_X_MINBLOCKS 1
#endif
#ifndef FVNA_Y_MINBLOCKS
#define FVNA_Y_MINBLOCKS 4    // 128 registers: 16 warps per SM (measured 25 % faster than 12)
#endif
#define FVNA_PRAGMA(x) _Pragma(#x)
#define FVNA_UNROLL(n) FVNA_PRAGMA(unroll n)

namespace fvna {

// ---------------------------------------------------------------------------
// cp.async (Ampere+ asynchronous global->shared copies, cache-all variant)
// ---------------------------------------------------------------------------
template <int BYTES> __device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(BYTES));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---------------------------------------------------------------------------
// Border handling: value of cell (gx, gy) of the state `q`, with every index
// outside the domain mapped by the border rule of its side.  x1 is mapped
// first, then x2 (a ghost column takes the x2 border of the column it maps
// to).  Reflection negates the normal momentum; driven borders evaluate the
// analytic value at the ghost-cell centre at time t.  Indices are clamped to
// the widest halo first, so periodic and mirror maps stay inside the domain
// for n >= 3.
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void load_mapped(const DomDev &D, const typename P::T *const q[3],
                                            int gx, int gy, double t, double dx,
                                            typename P::T out[3]) {
  typedef typename P::T T;
  const int nx = D.nx, ny = D.ny;
  bool flipx = false, flipy = false;
  int cx = gx, cy = gy;
  if (gx < 0 || gx >= nx) {
    if (gx > nx + HALO_Y - 1) gx = nx + HALO_Y - 1;
    int side = gx < 0 ? 0 : 1;
    int bc = D.bc[side];
    double xc = D.x0 + (gx + 0.5) * dx;
    double yc = D.y0 + (gy + 0.5) * dx;
    if (bc == BC_TAYLOR || (bc == BC_HIFU && side == 0 && yc >= 0.0 && yc <= D.aperture)) {
      if (bc == BC_HIFU && D.drive && gy >= 0 && gy < ny) {   // evaluated once per step
        const T *dv = (const T *)D.drive;
        size_t o = (size_t)(-1 - gx) * ny + gy, ps = (size_t)HALO_Y * ny;
        out[0] = dv[o]; out[1] = dv[ps + o]; out[2] = dv[2 * ps + o];
        return;
      }
      double v[3];
      if (bc == BC_TAYLOR) P::taylor(D, xc, yc, t, v); else P::hifu(D, xc, yc, t, v);
      out[0] = (T)v[0]; out[1] = (T)v[1]; out[2] = (T)v[2];
      return;
    }
    if (bc == BC_PERIODIC) cx = side == 0 ? gx + nx : gx - nx;
    else if (bc == BC_REFLECT) { cx = side == 0 ? -1 - gx : 2 * nx - 1 - gx; flipx = true; }
    else cx = side == 0 ? 0 : nx - 1;
  }
  if (gy < 0 || gy >= ny) {
    if (gy > ny + HALO_Y - 1) gy = ny + HALO_Y - 1;
    int side = gy < 0 ? 0 : 1;
    int bc = D.bc[2 + side];
    if (bc == BC_TAYLOR) {
      double v[3];
      P::taylor(D, D.x0 + (cx + 0.5) * dx, D.y0 + (gy + 0.5) * dx, t, v);
      out[0] = (T)v[0]; out[1] = flipx ? -(T)v[1] : (T)v[1]; out[2] = (T)v[2];
      return;
    }
    if (bc == BC_PERIODIC) cy = side == 0 ? gy + ny : gy - ny;
    else if (bc == BC_REFLECT) { cy = side == 0 ? -1 - gy : 2 * ny - 1 - gy; flipy = true; }
    else cy = side == 0 ? 0 : ny - 1;
  }
  size_t off = (size_t)cy * D.pitch + cx;
  T v0 = q[0][off], v1 = q[1][off], v2 = q[2][off];
  out[0] = v0;
  out[1] = flipx ? -v1 : v1;
  out[2] = flipy ? -v2 : v2;
}

// Is cell (gx, gy) a driven x1 ghost (its value is analytic, not mapped)?
__device__ __forceinline__ bool x_driven(const DomDev &D, int gx, int gy, double dx) {
  if (gx >= 0 && gx < D.nx) return false;
  int side = gx < 0 ? 0 : 1;
  int bc = D.bc[side];
  if (bc == BC_TAYLOR) return true;
  if (bc == BC_HIFU && side == 0) {
    double yc = D.y0 + (gy + 0.5) * dx;
    return yc >= 0.0 && yc <= D.aperture;
  }
  return false;
}

// ---------------------------------------------------------------------------
// The line march shared by both sweeps.  Cells c = 0..ncells-1 come from
// src.get(c, a, b, cc); interface k (1..ncells-1) lies between cells k-1
// and k; flux data exist for k = 2..ncells-2 and cells 2..ncells-3 are
// updated and handed to sink.put(c, a, b, cc).  Faces k in [klo, khi] count
// towards max|s|; interfaces in [nlo, nhi] towards the non-real flag.
// ---------------------------------------------------------------------------
// Running max of |s| kept as the bit pattern of |s|: for non-negative IEEE
// values the pattern orders like an unsigned integer and a NaN (positive
// sign) sorts above +inf, so the max cannot hide a NaN.  |s3| = |u| never
// exceeds max(|s1|, |s2|) = max(|u + c|, |u - c|) for c >= 0 (rounding is
// monotone), so two families suffice.
template <class T> struct SpeedBits;
template <> struct SpeedBits<float> {
  typedef unsigned int U;
  __device__ static __forceinline__ U bits(float s) { return __float_as_uint(s) & 0x7fffffffu; }
  __device__ static __forceinline__ double value(U b) { return (double)__uint_as_float(b); }
  __device__ static __forceinline__ U warp_max(U b) { return __reduce_max_sync(0xffffffffu, b); }
};
template <> struct SpeedBits<double> {
  typedef unsigned long long U;
  __device__ static __forceinline__ U bits(double s) {
    return (unsigned long long)__double_as_longlong(s) & 0x7fffffffffffffffull;
  }
  __device__ static __forceinline__ double value(U b) { return __longlong_as_double((long long)b); }
  __device__ static __forceinline__ U warp_max(U b) {
    for (int o = 16; o > 0; o >>= 1) {
      U v = __shfl_xor_sync(0xffffffffu, b, o);
      b = v > b ? v : b;
    }
    return b;
  }
};
template <class T>
__device__ __forceinline__ void speed_max(typename SpeedBits<T>::U &m, const Iface<T> &I) {
  typename SpeedBits<T>::U b0 = SpeedBits<T>::bits(I.s0), b1 = SpeedBits<T>::bits(I.s1);
  m = b0 > m ? b0 : m;
  m = b1 > m ? b1 : m;
}

// Interfaces in [glo, ghi] get the first-order flux (no correction term).
template <class T> __device__ __forceinline__ void first_order(FluxData<T> &f) {
  f.F[0] = T(0);
  f.F[1] = T(0);
  f.F[2] = T(0);
}

template <class P, int LIM, bool COMP, class Src, class Sink>
__device__ __forceinline__ void march(Src &src, Sink &sink, int ncells, typename P::T beta2,
                                      typename P::T lam, int klo, int khi, int nlo, int nhi,
                                      typename SpeedBits<typename P::T>::U &smax, bool &nonreal,
                                      int glo = 1, int ghi = 0) {
  typedef typename P::T T;
  T a0, b0, c0;        // cell c-2 (old)
  T a1, b1, c1;        // cell c-1 (old)
  T zb1, zc1;          // z of cell c-1
  Iface<T> Ia, Ib, Ic; // interfaces c-2, c-1, c
  FluxData<T> Fl, Fr;  // flux data of the left and right faces of cell c-2
  {
    T a, b, cc;
    src.get(0, a, b, cc);
    T r = P::rq1(a);
    a1 = a; b1 = b; c1 = cc; zb1 = b * r; zc1 = cc * r;
  }
  // cells 1..3: interfaces 1..3 and the flux data of interface 2
#pragma unroll
  for (int c = 1; c <= 3; c++) {
    T a, b, cc;
    src.get(c, a, b, cc);
    T r = P::rq1(a);
    T zb = b * r, zc = cc * r;
    Iface<T> I;
    bool nr = roe(P(), beta2, a1, b1, c1, zb1, zc1, a, b, cc, zb, zc, I);
    if (c >= nlo && c <= nhi) nonreal |= nr;
    a0 = a1; b0 = b1; c0 = c1;
    a1 = a; b1 = b; c1 = cc; zb1 = zb; zc1 = zc;
    if (c == 1) Ia = I;
    if (c == 2) Ib = I;
    if (c == 3) Ic = I;
  }
  flux_data<LIM, T>(Ib, Ia, Ic, lam, Fl);
  if (2 >= glo && 2 <= ghi) first_order(Fl);
  if (2 >= klo && 2 <= khi) speed_max<T>(smax, Ib);
  Ia = Ib;
  Ib = Ic;
  // now a0.. = cell 2, a1.. = cell 3
#if FVNA_MARCH_UNROLL > 0
  FVNA_UNROLL(FVNA_MARCH_UNROLL)
#endif
  for (int c = 4; c < ncells; c++) {
    T a, b, cc;
    src.get(c, a, b, cc);
    T r = P::rq1(a);
    T zb = b * r, zc = cc * r;
    bool nr = roe(P(), beta2, a1, b1, c1, zb1, zc1, a, b, cc, zb, zc, Ic);
    if (c >= nlo && c <= nhi) nonreal |= nr;
    // interface c-1 is the right face of cell c-2
    flux_data<LIM, T>(Ib, Ia, Ic, lam, Fr);
    if (c - 1 >= glo && c - 1 <= ghi) first_order(Fr);
    if (c - 1 >= klo && c - 1 <= khi) speed_max<T>(smax, Ib);
    T na = cell_update<COMP>(P(), a0, Fr.am[0], Fl.ap[0], Fr.F[0], Fl.F[0], lam);
    T nb = cell_update<COMP>(P(), b0, Fr.am[1], Fl.ap[1], Fr.F[1], Fl.F[1], lam);
    T nc = cell_update<COMP>(P(), c0, Fr.am[2], Fl.ap[2], Fr.F[2], Fl.F[2], lam);
    sink.put(c - 2, na, nb, nc);
    Ia = Ib;
    Ib = Ic;
    Fl = Fr;
    a0 = a1; b0 = b1; c0 = c1;
    a1 = a; b1 = b; c1 = cc; zb1 = zb; zc1 = zc;
  }
}

// The same traversal with the sweep switched off: cells pass through unchanged.
template <class P, class Src, class Sink>
__device__ __forceinline__ void march_copy(Src &src, Sink &sink, int ncells) {
  typedef typename P::T T;
  for (int c = 0; c < ncells; c++) {
    T a, b, cc;
    src.get(c, a, b, cc);
    if (c >= 2 && c <= ncells - 3) sink.put(c, a, b, cc);
  }
}

// ---------------------------------------------------------------------------
// x1 sweep
// ---------------------------------------------------------------------------
template <class T> struct SmemRowSrc {
  const T *row;
  int fstride;
  __device__ __forceinline__ void get(int c, T &a, T &b, T &cc) const {
    a = row[c];
    b = row[fstride + c];
    cc = row[2 * fstride + c];
  }
};
template <class T> struct SmemRowSink {
  T *row;
  int fstride, chi;
  __device__ __forceinline__ void put(int c, T a, T b, T cc) const {
    if (c <= chi) {
      row[c] = a;
      row[fstride + c] = b;
      row[2 * fstride + c] = cc;
    }
  }
};

template <class P, int TX, int LIM, bool COMP>
__global__ void __launch_bounds__(128, FVNA_X_MINBLOCKS) k_sweep_x(StepArgs A) {
  typedef typename P::T T;
  constexpr int NC = TX + 2 * HALO_X;
  constexpr int PITCH = NC + 1;             // odd: a column read by 32 lanes is conflict-free
  constexpr int FS = XROWS * PITCH;         // field stride in shared memory
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T *sm = reinterpret_cast<T *>(smem_raw) + (size_t)warp * 3 * FS;
  const int wstride = gridDim.x * (blockDim.x >> 5);
  const T beta2 = (T)(2.0 * (A.beta - 1.0));
  const bool xsweep = (A.sweeps & 1) != 0;

  for (int w = blockIdx.x * (blockDim.x >> 5) + warp; w < A.ntiles; w += wstride) {
    const Tile tl = A.tiles[w];
    const DomDev &D = A.doms[tl.dom];
    DomScal *S = A.scal + tl.dom;
    if (S->done) continue;
    const double t = S->t;
    // dt/dx, halved (exactly) for the two x1 sweeps of a Strang step
    const T lam = (P::pert ? (T)S->lam32 : (T)S->lam) * (A.x_half ? (T)0.5 : (T)1);
    const int nx = D.nx, ny = D.ny;
    const T *qi[3] = {(const T *)D.qa[0], (const T *)D.qa[1], (const T *)D.qa[2]};
    T *qo[3] = {(T *)D.qb[0], (T *)D.qb[1], (T *)D.qb[2]};
    const bool interior = tl.x0 - HALO_X >= 0 && tl.x0 + TX + HALO_X <= nx;

    // load the tile and its halo
    for (int e = lane; e < XROWS * NC; e += 32) {
      int r = e / NC, c = e - r * NC;
      int gy = tl.y0 + r;
      if (gy >= ny) continue;
      int gx = tl.x0 - HALO_X + c;
      T *dst = sm + r * PITCH + c;
      if (interior || (gx >= 0 && gx < nx)) {
        size_t off = (size_t)gy * D.pitch + gx;
        cp_async<sizeof(T)>(dst, qi[0] + off);
        cp_async<sizeof(T)>(dst + FS, qi[1] + off);
        cp_async<sizeof(T)>(dst + 2 * FS, qi[2] + off);
      } else {
        T v[3];
        load_mapped<P>(D, qi, gx, gy, t, A.dx, v);
        dst[0] = v[0];
        dst[FS] = v[1];
        dst[2 * FS] = v[2];
      }
    }
    cp_commit();
    cp_wait<0>();
    __syncwarp();

    typename SpeedBits<T>::U smax = 0;
    bool nonreal = false;
    // with the x1 sweep off the tile is stored unchanged
    if (xsweep && tl.y0 + lane < ny) {
      T *row = sm + lane * PITCH;
      SmemRowSrc<T> src{row, FS};
      SmemRowSink<T> sink{row, FS, nx - tl.x0 + HALO_X - 1};
      int khi = min(TX + HALO_X, nx - tl.x0 + HALO_X);
      int nhi = min(NC - 1, nx + 1 - (tl.x0 - HALO_X));
      march<P, LIM, COMP>(src, sink, NC, beta2, lam, HALO_X, khi, 1, nhi, smax, nonreal);
    }
    __syncwarp();

    // store the updated cells
    for (int e = lane; e < XROWS * TX; e += 32) {
      int r = e / TX, c = e - r * TX;
      int gy = tl.y0 + r, gx = tl.x0 + c;
      if (gy < ny && gx < nx) {
        size_t off = (size_t)gy * D.pitch + gx;
        const T *s = sm + r * PITCH + c + HALO_X;
        qo[0][off] = s[0];
        qo[1][off] = s[FS];
        qo[2][off] = s[2 * FS];
      }
    }
    smax = SpeedBits<T>::warp_max(smax);
    int nr = warp_or(nonreal ? 1 : 0);
    if (lane == 0) {
      atomic_max_speed(&S->smax_bits, SpeedBits<T>::value(smax));
      if (nr) atomicOr(&S->status_bits, ST_NONREAL);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// x2 sweep + source
// ---------------------------------------------------------------------------
template <class P, int RING> struct RingSrc {
  typedef typename P::T T;
  T *ring;                 // RING slots x 3 fields x 32 lanes
  const T *const *q;
  const DomDev *D;
  int lane, gx, col, y0, ncells;
  bool plain_col;          // column inside the domain or a plain (unflipped, undriven) map
  double t, dx;

  __device__ __forceinline__ void issue(int c) {
    if (c < ncells) {
      int gy = y0 - HALO_Y + c;
      T *slot = ring + (c & (RING - 1)) * 96 + lane;
      if (plain_col && gy >= 0 && gy < D->ny) {
        size_t off = (size_t)gy * D->pitch + col;
        cp_async<sizeof(T)>(slot, q[0] + off);
        cp_async<sizeof(T)>(slot + 32, q[1] + off);
        cp_async<sizeof(T)>(slot + 64, q[2] + off);
      } else {
        T v[3];
        load_mapped<P>(*D, q, gx, gy, t, dx, v);
        slot[0] = v[0];
        slot[32] = v[1];
        slot[64] = v[2];
      }
    }
    cp_commit();
  }
  // march order of the x2 sweep: (q1, q3, q2)
  __device__ __forceinline__ void get(int c, T &a, T &b, T &cc) {
    issue(c + RING - 1);
    cp_wait<RING - 1>();
    const T *slot = ring + (c & (RING - 1)) * 96 + lane;
    a = slot[0];
    cc = slot[32];
    b = slot[64];
  }
};

// Warp sum of (partial sum, rounding error) pairs: binary64 adds it directly;
// binary32 combines the pairs with two-sums and converts once on the result.
__device__ __forceinline__ double warp_sum_pair(double s, double e) { return warp_sum(s + e); }
__device__ __forceinline__ double warp_sum_pair(float s, float e) {
  for (int o = 16; o > 0; o >>= 1) {
    float so = __shfl_xor_sync(0xffffffffu, s, o);
    float eo = __shfl_xor_sync(0xffffffffu, e, o);
    float t = s + so;
    float bb = t - s;
    e = e + eo + ((s - (t - bb)) + (so - bb));
    s = t;
  }
  return (double)s + (double)e;
}

template <class P> struct YSink {
  typedef typename P::T T;
  const DomDev *D;
  T *const *qo;
  int lane, gx, y0, tile_y;
  bool upd_lane, xdrv, source, axi;
  double t, dx, dt;
  T coef, dtT;
  // post-x2-sweep row e-1 and the velocities z of rows e-1, e-2
  T qp0, qp1, qp2, zp2, zp3, zpp2, zpp3;
  // per-lane budget partial sums; in binary32 with their rounding errors
  // (two-sum), so the binary64 totals keep the precision of binary64 sums
  T bud[3], bude[3];

  __device__ __forceinline__ void acc(int k, T x) {
    if (!P::pert) {
      bud[k] += x;
      return;
    }
    T s = bud[k] + x;
    T bb = s - bud[k];
    bude[k] += (bud[k] - (s - bb)) + (x - bb);
    bud[k] = s;
  }

  __device__ __forceinline__ void zof(T q0, T q1, T q2, T &z2, T &z3) const {
    T r = P::rq1(q0);
    z2 = q1 * r;
    z3 = q2 * r;
  }
  __device__ __forceinline__ void analytic(int bc, int cx, int gy, T o[3]) const {
    if (bc == BC_HIFU && D->drive && cx < 0 && gy >= 0 && gy < D->ny) {
      const T *dv = (const T *)D->drive;
      size_t of = (size_t)(-1 - cx) * D->ny + gy, ps = (size_t)HALO_Y * D->ny;
      o[0] = dv[of]; o[1] = dv[ps + of]; o[2] = dv[2 * ps + of];
      return;
    }
    double v[3];
    double xc = D->x0 + (cx + 0.5) * dx, yc = D->y0 + (gy + 0.5) * dx;
    if (bc == BC_TAYLOR) P::taylor(*D, xc, yc, t, v); else P::hifu(*D, xc, yc, t, v);
    o[0] = (T)v[0]; o[1] = (T)v[1]; o[2] = (T)v[2];
  }

  // a, b, cc in march order (q1, q3, q2)
  __device__ __forceinline__ void put(int c, T a, T b, T cc) {
    const int e = y0 - HALO_Y + c;
    const int ny = D->ny;
    T q0 = a, q1 = cc, q2 = b;
    if (xdrv && e >= 0 && e < ny && x_driven(*D, gx, e, dx)) {
      T v[3];
      analytic(D->bc[gx < 0 ? 0 : 1], gx, e, v);
      q0 = v[0]; q1 = v[1]; q2 = v[2];
    }
    if (e == ny) {  // x2-high ghost row from the post-sweep row ny-1
      int bc = D->bc[3];
      if (bc == BC_EXTRAP || bc == BC_HIFU) { q0 = qp0; q1 = qp1; q2 = qp2; }
      else if (bc == BC_REFLECT) { q0 = qp0; q1 = qp1; q2 = -qp2; }
      else if (bc == BC_TAYLOR) {
        T v[3];
        analytic(BC_TAYLOR, gx, e, v);
        q0 = v[0]; q1 = v[1]; q2 = v[2];
      }
    }
    T z2, z3;
    zof(q0, q1, q2, z2, z3);
    if (e == 0 && y0 == 0) {  // x2-low ghost row from the post-sweep row 0
      int bc = D->bc[2];
      if (bc == BC_EXTRAP || bc == BC_HIFU) { zp2 = z2; zp3 = z3; }
      else if (bc == BC_REFLECT) { zp2 = z2; zp3 = -z3; }
      else if (bc == BC_TAYLOR) {
        T v[3];
        analytic(BC_TAYLOR, gx, -1, v);
        zof(v[0], v[1], v[2], zp2, zp3);
      }
    }
    // source on row e-1 (the x1 neighbours come from the adjacent lanes)
    const int er = e - 1;
    T w2 = __shfl_up_sync(0xffffffffu, zp2, 1);
    T e2 = __shfl_down_sync(0xffffffffu, zp2, 1);
    T w3 = __shfl_up_sync(0xffffffffu, zp3, 1);
    T e3 = __shfl_down_sync(0xffffffffu, zp3, 1);
    if (c >= 3 && er >= y0 && er < y0 + tile_y && er < ny && upd_lane) {
      T o0 = qp0, o1 = qp1, o2 = qp2;
      if (source) {
        if (!axi) {
          T L2 = (w2 + e2) + (zpp2 + z2) - T(4) * zp2;
          T L3 = (w3 + e3) + (zpp3 + z3) - T(4) * zp3;
          o1 = o1 + coef * L2;
          o2 = o2 + coef * L3;
        } else {
          T r = P::pert ? (T)D->y0 + ((T)er + T(0.5)) * (T)dx : (T)(D->y0 + (er + 0.5) * dx);
          T L2 = (w2 + e2) + (zpp2 + z2) - T(4) * zp2 + (z2 - zpp2) * ((T)dx / (T(2) * r));
          T L3 = (w3 + e3) + (zpp3 + z3) - T(4) * zp3 + (z3 - zpp3) * ((T)dx / (T(2) * r)) -
                 zp3 * ((T)dx * (T)dx / (r * r));
          T g1 = qp2 / r;
          T g2 = zp2 * zp3 / r;
          T g3 = zp3 * zp3 / r;
          o0 = o0 - dtT * g1;
          o1 = o1 + coef * L2 - dtT * g2;
          o2 = o2 + coef * L3 - dtT * g3;
        }
      }
      size_t off = (size_t)er * D->pitch + gx;
      qo[0][off] = o0;
      qo[1][off] = o1;
      qo[2][off] = o2;
      acc(0, P::pert ? o0 : o0 - T(1));
      acc(1, o1);
      acc(2, o2);
    }
    qp0 = q0; qp1 = q1; qp2 = q2;
    zpp2 = zp2; zpp3 = zp3;
    zp2 = z2; zp3 = z3;
  }
};

template <class P, int RING, int LIM, bool COMP>
__global__ void __launch_bounds__(128, FVNA_Y_MINBLOCKS) k_sweep_y(StepArgs A) {
  typedef typename P::T T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T *ring = reinterpret_cast<T *>(smem_raw) + (size_t)warp * RING * 96;
  const int wstride = gridDim.x * (blockDim.x >> 5);
  const T beta2 = (T)(2.0 * (A.beta - 1.0));
  const bool ysweep = (A.sweeps & 2) != 0;
  const bool source = (A.sweeps & 4) != 0;

  for (int w = blockIdx.x * (blockDim.x >> 5) + warp; w < A.ntiles; w += wstride) {
    const Tile tl = A.tiles[w];
    const DomDev &D = A.doms[tl.dom];
    DomScal *S = A.scal + tl.dom;
    if (S->done) continue;
    const double dt = S->dt, t = S->t;
    const T lam = P::pert ? (T)S->lam32 : (T)S->lam;
    const int nx = D.nx, ny = D.ny;
    const int TY = A.tile_y;
    const int ncells = TY + 2 * HALO_Y;
    // input: the planes written by the x1 sweep (never the planes written here)
    const T *qi[3] = {(const T *)D.qb[0], (const T *)D.qb[1], (const T *)D.qb[2]};
    T *qo[3] = {(T *)D.qa[0], (T *)D.qa[1], (T *)D.qa[2]};

    int gx = tl.x0 - 1 + lane;
    if (gx > nx) gx = nx;  // lanes past the x1-high ghost column duplicate it
    // column map of this lane
    int col = gx;
    bool plain = true, xdrv = false;
    if (gx < 0 || gx >= nx) {
      int side = gx < 0 ? 0 : 1;
      int bc = D.bc[side];
      if (bc == BC_PERIODIC) col = side == 0 ? gx + nx : gx - nx;
      else if (bc == BC_REFLECT) { col = side == 0 ? 0 : nx - 1; plain = false; }
      // driven ghost columns march the edge column (as extrapolation does)
      // and replace the swept values by the analytic ones where driven
      else if (bc == BC_TAYLOR) { col = side == 0 ? 0 : nx - 1; xdrv = true; }
      else if (bc == BC_HIFU && side == 0) { col = 0; xdrv = true; }
      else col = side == 0 ? 0 : nx - 1;
    }
    const bool upd_lane = lane >= 1 && lane <= YCOLS && gx >= 0 && gx < nx && gx == tl.x0 - 1 + lane;

    RingSrc<P, RING> src;
    src.ring = ring; src.q = qi; src.D = &D; src.lane = lane; src.gx = gx; src.col = col;
    src.y0 = tl.y0; src.ncells = ncells; src.plain_col = plain; src.t = t; src.dx = A.dx;
#pragma unroll
    for (int c = 0; c < RING - 1; c++) src.issue(c);

    YSink<P> sink;
    sink.D = &D; sink.qo = qo; sink.lane = lane; sink.gx = gx; sink.y0 = tl.y0;
    sink.tile_y = TY; sink.upd_lane = upd_lane; sink.xdrv = xdrv; sink.source = source;
    sink.axi = A.geometry == 1; sink.t = t; sink.dx = A.dx; sink.dt = dt;
    sink.coef = P::pert ? (T)S->coef32 : (T)S->coef;
    sink.dtT = P::pert ? (T)S->dt32 : (T)dt;
    sink.qp0 = sink.qp1 = sink.qp2 = T(0);
    sink.zp2 = sink.zp3 = sink.zpp2 = sink.zpp3 = T(0);
    for (int k = 0; k < 3; k++) sink.bud[k] = sink.bude[k] = T(0);

    typename SpeedBits<T>::U smax = 0;
    bool nonreal = false;
    // faces of this tile's cells (k = 3 is face y0), and the interfaces the
    // reference sweep computes (faces -1..ny+1), for in-domain lanes only
    int klo = HALO_Y, khi = min(TY + HALO_Y, ny - tl.y0 + HALO_Y);
    int nlo = max(1, 2 - tl.y0), nhi = ny + 4 - tl.y0;
    if (!upd_lane) { klo = 1; khi = 0; nlo = 1; nhi = 0; }
    // axisymmetric form: first-order flux on the radial faces at r = 0 and
    // r = dx (faces 0 and 1, local interfaces 3 and 4 of the first row tile)
    int glo = 1, ghi = 0;
    if (A.geometry == 1 && D.y0 == 0.0 && tl.y0 == 0) { glo = HALO_Y; ghi = HALO_Y + AXIS_FACES - 1; }
    if (ysweep)
      march<P, LIM, COMP>(src, sink, ncells, beta2, lam, klo, khi, nlo, nhi, smax, nonreal, glo,
                          ghi);
    else
      march_copy<P>(src, sink, ncells);
    cp_wait<0>();
    __syncwarp();

    smax = SpeedBits<T>::warp_max(smax);
    int nr = warp_or(nonreal ? 1 : 0);
    double b0 = warp_sum_pair(sink.bud[0], sink.bude[0]);
    double b1 = warp_sum_pair(sink.bud[1], sink.bude[1]);
    double b2 = warp_sum_pair(sink.bud[2], sink.bude[2]);
    if (lane == 0) {
      atomic_max_speed(&S->smax_bits, SpeedBits<T>::value(smax));
      if (nr) atomicOr(&S->status_bits, ST_NONREAL);
      atomicAdd(&S->budget_acc[0], b0);
      atomicAdd(&S->budget_acc[1], b1);
      atomicAdd(&S->budget_acc[2], b2);
    }
  }
}

// ---------------------------------------------------------------------------
// HIFU drive of the current step (eq. hifuBC) at the ghost columns -1..-3 of
// every row inside the aperture, evaluated once per step instead of in every
// load (the drive costs sin/exp in binary64 per value).
// ---------------------------------------------------------------------------
template <class P>
__global__ void k_drive(StepArgs A, int dom, int always) {
  typedef typename P::T T;
  const DomDev &D = A.doms[dom];
  const DomScal *S = A.scal + dom;
  if ((S->done && !always) || !D.drive) return;
  const int n = HALO_Y * D.ny;
  T *dv = (T *)D.drive;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int layer = e / D.ny, row = e - layer * D.ny;
    int gx = -1 - layer;
    double xc = D.x0 + (gx + 0.5) * A.dx, yc = D.y0 + (row + 0.5) * A.dx;
    double v[3] = {0.0, 0.0, 0.0};
    if (yc >= 0.0 && yc <= D.aperture) P::hifu(D, xc, yc, S->t, v);
    dv[e] = (T)v[0];
    dv[n + e] = (T)v[1];
    dv[2 * n + e] = (T)v[2];
  }
}

// ---------------------------------------------------------------------------
// Speed-only pass over all faces of a domain (the first dt, section 4).
// ---------------------------------------------------------------------------
template <class P>
__global__ void k_speeds(StepArgs A, int dom, int use_b) {
  typedef typename P::T T;
  const DomDev &D = A.doms[dom];
  DomScal *S = A.scal + dom;
  const T beta2 = (T)(2.0 * (A.beta - 1.0));
  const T *q[3];
  for (int k = 0; k < 3; k++) q[k] = (const T *)(use_b ? D.qb[k] : D.qa[k]);
  const long long nxf = (long long)(D.nx + 1) * D.ny;
  const long long nyf = (long long)D.nx * (D.ny + 1);
  typename SpeedBits<T>::U smax = 0;
  bool nonreal = false;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nxf + nyf;
       f += (long long)gridDim.x * blockDim.x) {
    T L[3], R[3];
    Iface<T> I;
    bool nr;
    if (f < nxf) {
      int j = (int)(f / (D.nx + 1)), i = (int)(f - (long long)j * (D.nx + 1));
      load_mapped<P>(D, q, i - 1, j, S->t, A.dx, L);
      load_mapped<P>(D, q, i, j, S->t, A.dx, R);
      T rl = P::rq1(L[0]), rr = P::rq1(R[0]);
      nr = roe(P(), beta2, L[0], L[1], L[2], L[1] * rl, L[2] * rl, R[0], R[1], R[2], R[1] * rr,
               R[2] * rr, I);
    } else {
      long long g = f - nxf;
      int j = (int)(g / D.nx), i = (int)(g - (long long)j * D.nx);
      load_mapped<P>(D, q, i, j - 1, S->t, A.dx, L);
      load_mapped<P>(D, q, i, j, S->t, A.dx, R);
      T rl = P::rq1(L[0]), rr = P::rq1(R[0]);
      nr = roe(P(), beta2, L[0], L[2], L[1], L[2] * rl, L[1] * rl, R[0], R[2], R[1], R[2] * rr,
               R[1] * rr, I);
    }
    nonreal |= nr;
    speed_max<T>(smax, I);
  }
  smax = SpeedBits<T>::warp_max(smax);
  int nr = warp_or(nonreal ? 1 : 0);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_speed(&S->smax_bits, SpeedBits<T>::value(smax));
    if (nr) atomicOr(&S->status_bits, ST_NONREAL);
  }
}

// ---------------------------------------------------------------------------
// State conversion between the caller's binary64 total variables and the
// stored form.
// ---------------------------------------------------------------------------
template <class P>
__global__ void k_import(DomDev D, const double *q0) {
  typedef typename P::T T;
  const long long n = (long long)D.nx * D.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int j = (int)(c / D.nx), i = (int)(c - (long long)j * D.nx);
    size_t off = (size_t)j * D.pitch + i;
    double a = q0[c], b = q0[n + c], cc = q0[2 * n + c];
    ((T *)D.qa[0])[off] = P::pert ? (T)(a - 1.0) : (T)a;
    ((T *)D.qa[1])[off] = (T)b;
    ((T *)D.qa[2])[off] = (T)cc;
  }
}

// what: 0 = q (3 planes, total variables), 1 = q1 - 1, 2 = q1 - 1 of row 0
template <class P>
__global__ void k_export(DomDev D, double *out, int what) {
  typedef typename P::T T;
  const long long n = what == 2 ? (long long)D.nx : (long long)D.nx * D.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int j = (int)(c / D.nx), i = (int)(c - (long long)j * D.nx);
    size_t off = (size_t)j * D.pitch + i;
    double a = (double)((const T *)D.qa[0])[off];
    if (what >= 1) {
      out[c] = P::pert ? a : a - 1.0;
    } else {
      out[c] = P::pert ? 1.0 + a : a;
      out[n + c] = (double)((const T *)D.qa[1])[off];
      out[2 * n + c] = (double)((const T *)D.qa[2])[off];
    }
  }
}

// ---------------------------------------------------------------------------
// Moving domain (section 4: in the second stage of a run the domain moves
// with the wave).  The window moves by (kx, ky) whole cells: new cell (i, j)
// takes old cell (i + kx, j + ky).  A cell with no old counterpart comes in
// through a border and takes what that border's rule gives at the domain's
// current time: the Taylor shock its analytic value (eq. OurTaylorS) at the
// new cell centre; periodic the wrapped old cell; every other rule the
// nearest old cell.  Through a corner: the analytic value if either border
// is a Taylor border, else both rules in turn.  k_shift writes the moved
// state into the swept planes; k_shift_back copies it back and moves the
// corner of the device descriptor (the corner is only ever read from there).
// Coordinates are rounded operation by operation, so both precisions' units
// compute the same centres.
// ---------------------------------------------------------------------------
template <class P>
__global__ void k_shift(DomDev D, const DomDev *dd, int dom, const DomScal *S, int kx, int ky,
                        double dx) {
  typedef typename P::T T;
  const int nx = D.nx, ny = D.ny;
  const double t = S->t;
  D.x0 = dd[dom].x0;
  D.y0 = dd[dom].y0;
  const double x0n = __dadd_rn(D.x0, __dmul_rn((double)kx, dx));
  const double y0n = __dadd_rn(D.y0, __dmul_rn((double)ky, dx));
  const long long n = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    const size_t off = (size_t)j * D.pitch + i;
    int si = i + kx, sj = j + ky;
    const bool ox = si < 0 || si >= nx, oy = sj < 0 || sj >= ny;
    const int bx = D.bc[si < 0 ? 0 : 1], by = D.bc[sj < 0 ? 2 : 3];
    if ((ox && bx == BC_TAYLOR) || (oy && by == BC_TAYLOR)) {
      double v[3];
      P::taylor(D, __dadd_rn(x0n, __dmul_rn((double)i + 0.5, dx)),
                __dadd_rn(y0n, __dmul_rn((double)j + 0.5, dx)), t, v);
      for (int k = 0; k < 3; k++) ((T *)D.qb[k])[off] = (T)v[k];
      continue;
    }
    if (ox) si = bx == BC_PERIODIC ? (si < 0 ? si + nx : si - nx) : (si < 0 ? 0 : nx - 1);
    if (oy) sj = by == BC_PERIODIC ? (sj < 0 ? sj + ny : sj - ny) : (sj < 0 ? 0 : ny - 1);
    const size_t so = (size_t)sj * D.pitch + si;
    for (int k = 0; k < 3; k++) ((T *)D.qb[k])[off] = ((const T *)D.qa[k])[so];
  }
}
template <class P>
__global__ void k_shift_back(DomDev D, DomDev *dd, int dom, int kx, int ky, double dx) {
  typedef typename P::T T;
  const long long n = (long long)D.nx * D.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / D.nx), i = (int)(c - (long long)j * D.nx);
    const size_t off = (size_t)j * D.pitch + i;
    for (int k = 0; k < 3; k++) ((T *)D.qa[k])[off] = ((const T *)D.qb[k])[off];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dd[dom].x0 = __dadd_rn(dd[dom].x0, __dmul_rn((double)kx, dx));
    dd[dom].y0 = __dadd_rn(dd[dom].y0, __dmul_rn((double)ky, dx));
  }
}

// Device Roe solver on host-supplied pairs (binary64 total variables in).
template <class P>
__global__ void k_riemann(double beta, int n, const double *qL, const double *qR, double *s,
                          double *W, double *am, double *ap, int *nonreal) {
  typedef typename P::T T;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  T L[3], R[3];
  for (int c = 0; c < 3; c++) {
    L[c] = (T)(c == 0 && P::pert ? qL[3 * k] - 1.0 : qL[3 * k + c]);
    R[c] = (T)(c == 0 && P::pert ? qR[3 * k] - 1.0 : qR[3 * k + c]);
  }
  T rl = P::rq1(L[0]), rr = P::rq1(R[0]);
  Iface<T> I;
  bool nr = roe(P(), (T)(2.0 * (beta - 1.0)), L[0], L[1], L[2], L[1] * rl, L[2] * rl, R[0], R[1],
                R[2], R[1] * rr, R[2] * rr, I);
  if (nr) atomicOr(nonreal, 1);
  FluxData<T> F;
  flux_data<LIM_NONE, T>(I, I, I, T(0), F);
  s[3 * k] = I.s0; s[3 * k + 1] = I.s1; s[3 * k + 2] = I.s2;
  for (int c = 0; c < 3; c++) {
    W[9 * k + c] = I.W0[c];
    W[9 * k + 3 + c] = I.W1[c];
    W[9 * k + 6 + c] = c == 2 ? (double)I.W2 : 0.0;
    am[3 * k + c] = F.am[c];
    ap[3 * k + c] = F.ap[c];
  }
}

}  // namespace fvna
