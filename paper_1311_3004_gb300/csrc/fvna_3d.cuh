// fvna_3d.cuh -- the three-dimensional form of the finite-volume step
// (arXiv 1311.3004: the equations of section 2 with a third velocity
// component, which the paper states carry over directly; the scheme of
// section 3 with a third directional sweep).  Included by one translation
// unit per precision:
//   fvna_3d64.cu  binary64 total variables (q1, q2, q3, q4), compiled with
//                 -fmad=false: every formula below is evaluated in the order
//                 of the definitions, so results match a plain binary64
//                 evaluation of the same definitions bit for bit;
//   fvna_3d32.cu  binary32 perturbation variables (q1 - 1, q2, q3, q4).
//
// One step: x1 sweep (state -> swept planes), x2 sweep (back), x3 sweep
// (again), source (back into the state), dt update.  Each sweep is eq. fv-hr
// on lines of the 4-component system with the entries permuted so that the
// normal momentum comes second; the Roe solver of section 3.2 gains the
// fourth component, which behaves as the third (a transverse family moving
// at u, eigenvectors r1, r2 with fourth components w (s1 - 2 Z2)/c and
// w (2 Z2 - s2)/c, w = Z4/Z1).
//
//   k3_sweep_x   x1 sweep: a warp holds 64 cells of one row, two per lane,
//                each lane solving the faces on the left of its cells and
//                exchanging neighbour faces by shuffles; 60 cells updated
//                per segment, coalesced two-element loads and stores.
//   k3_sweep_v   x2 or x3 sweep: the lanes hold 32 consecutive x1 columns and
//                march together along x2 (or x3) over TY cells plus two halo
//                cells at each end, loading and storing one coalesced row per
//                field and cell.
//   k3_source    forward Euler with the 7-point Laplacian of z = q/q1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fvna {
namespace d3 {

enum { B_PERIODIC = 0, B_EXTRAP = 1, B_REFLECT = 2 };
enum { L_MC = 0, L_NONE = 1, L_LW = 2 };
enum { S_NONREAL = 1, S_CFL = 2, S_NAN = 4 };

// One 3D domain: four field planes of pitch * ny * nz elements, x1 fastest.
struct Dom3 {
  int nx, ny, nz, pitch;
  long long plane;        // elements per field plane
  int bc[6];              // x1-low, x1-high, x2-low, x2-high, x3-low, x3-high
};

// Scalars that evolve on the device.
struct Scal3 {
  double t, dt, dt_cfl, dt_last, t_end, smax_last;
  double nu_min, nu_max, nu_mean, nu_m2;
  long long nu_count, step, steps_left;
  unsigned long long smax_bits;   // atomic max of |s| during the step (bit pattern)
  int status_bits, status, done, last, timed, pad;
  double lam, coef;               // dt/dx and dt delta / dx^2 of the step
  float lam32, coef32;
};

struct Args3 {
  Dom3 d;
  Scal3 *S;
  const void *in[4];      // planes read by the launch
  void *out[4];           // planes written by the launch
  double beta, delta, dx, nu_w, nu_max, dt_fixed;
  int limiter, comp, dir, tile;   // dir: 0 x1, 1 x2, 2 x3; tile: TY of the x2/x3 sweeps
};

// ---------------------------------------------------------------------------
// Border rules: index of cell g of a line of n cells, g outside [0, n) being a
// ghost cell, and whether the normal momentum flips sign.  Cells beyond the
// two ghost layers (the x1 sweep's last tile reads past the end of a short
// line) are clamped to the outer layer first: they only feed faces outside
// the domain, and the periodic and mirror maps stay inside [0, n) for n >= 3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int map_cell(int g, int n, int bclo, int bchi, bool &flip) {
  flip = false;
  if (g >= 0 && g < n) return g;
  g = g < -2 ? -2 : g > n + 1 ? n + 1 : g;
  if (g < 0) {
    if (bclo == B_PERIODIC) return g + n;
    if (bclo == B_REFLECT) { flip = true; return -1 - g; }
    return 0;
  }
  if (bchi == B_PERIODIC) return g - n;
  if (bchi == B_REFLECT) { flip = true; return 2 * n - 1 - g; }
  return n - 1;
}

// ---------------------------------------------------------------------------
// Precision: the stored first field is q1 (binary64) or q1 - 1 (binary32).
// ---------------------------------------------------------------------------
template <class T> struct Face4 {
  T s0, s1, u, a1, a2, a3, a4, r13, r23, r14, r24;
};

// 1/x in binary32: the hardware approximation refined by one Newton step
// r + r (1 - x r), within an ulp or so of the exact reciprocal and not
// biased to one side (the approximation alone errs one way)
__device__ __forceinline__ float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ double inv_q1(double a) { return 1.0 / a; }
__device__ __forceinline__ float inv_q1(float a) { return rcp_nr(1.0f + a); }

// Roe solver of one interface, binary64, in the order of the definitions.
// L, R = (q1, normal momentum, transverse 1, transverse 2); zL, zR = the
// velocities (q2, q3, q4)/q1 of the two cells in the same order.
__device__ __forceinline__ bool roe4(double beta, const double L[4], const double zL[3],
                                     const double R[4], const double zR[3], Face4<double> &F) {
  double Z1 = 0.5 * (L[0] + R[0]);
  double Z2 = 0.5 * (zL[0] + zR[0]);
  double Z3 = 0.5 * (zL[1] + zR[1]);
  double Z4 = 0.5 * (zL[2] + zR[2]);
  double Phi = 1.0 + 2.0 * (beta - 1.0) * (Z1 - 1.0);
  double rZ1 = 1.0 / Z1;
  double u = Z2 * rZ1;
  double v = Z3 * rZ1;
  double w = Z4 * rZ1;
  double D = u * u - 2.0 * Z2 * u + Phi;
  bool nonreal = D < 0.0;
  double c = sqrt(D);
  F.s0 = u + c;
  F.s1 = u - c;
  F.u = u;
  double rc = 1.0 / c;
  double h = 0.5 * rc;
  double d1 = R[0] - L[0];
  double d2 = R[1] - L[1];
  double d3 = R[2] - L[2];
  double d4 = R[3] - L[3];
  F.r13 = v * (F.s0 - 2.0 * Z2) * rc;
  F.r23 = v * (2.0 * Z2 - F.s1) * rc;
  F.r14 = w * (F.s0 - 2.0 * Z2) * rc;
  F.r24 = w * (2.0 * Z2 - F.s1) * rc;
  F.a1 = (d2 - F.s1 * d1) * h;
  F.a2 = (F.s0 * d1 - d2) * h;
  F.a3 = d3 - F.a1 * F.r13 - F.a2 * F.r23;
  F.a4 = d4 - F.a1 * F.r14 - F.a2 * F.r24;
  return nonreal;
}

// The same in binary32 perturbation form: Z1 - 1, D - 1 and c - 1 are carried
// as small numbers.  c - 1 = (D - 1) / (1 + sqrt(D)) keeps the relative
// precision of D - 1, so the approximate square root only touches it at the
// 1e-7 relative level, and the reciprocals take a Newton step (a one-signed
// error there would bias every wave speed).
__device__ __forceinline__ bool roe4(float beta, const float L[4], const float zL[3],
                                     const float R[4], const float zR[3], Face4<float> &F) {
  float Z1p = 0.5f * (L[0] + R[0]);
  float Z2 = 0.5f * (zL[0] + zR[0]);
  float Z3 = 0.5f * (zL[1] + zR[1]);
  float Z4 = 0.5f * (zL[2] + zR[2]);
  float rZ1 = rcp_nr(1.0f + Z1p);
  float u = Z2 * rZ1;
  float v = Z3 * rZ1;
  float w = Z4 * rZ1;
  float dm = u * u - 2.0f * Z2 * u + 2.0f * (beta - 1.0f) * Z1p;   // D - 1
  bool nonreal = dm < -1.0f;
  float D = 1.0f + dm;
  float e = dm * rcp_nr(fmaf(D, rsqrt_approx(D), 1.0f));           // c - 1
  float c = 1.0f + e;
  F.s0 = u + c;
  F.s1 = u - c;
  F.u = u;
  float rc = rcp_nr(c);
  float h = 0.5f * rc;
  float d1 = R[0] - L[0];
  float d2 = R[1] - L[1];
  float d3 = R[2] - L[2];
  float d4 = R[3] - L[3];
  F.r13 = v * (F.s0 - 2.0f * Z2) * rc;
  F.r23 = v * (2.0f * Z2 - F.s1) * rc;
  F.r14 = w * (F.s0 - 2.0f * Z2) * rc;
  F.r24 = w * (2.0f * Z2 - F.s1) * rc;
  F.a1 = (d2 - F.s1 * d1) * h;
  F.a2 = (F.s0 * d1 - d2) * h;
  F.a3 = d3 - F.a1 * F.r13 - F.a2 * F.r23;
  F.a4 = d4 - F.a1 * F.r14 - F.a2 * F.r24;
  return nonreal;
}

// Waves W[p][k] = a_p r_p of a face (family p, component k).
template <class T> __device__ __forceinline__ void waves(const Face4<T> &F, T W[4][4]) {
  W[0][0] = F.a1; W[0][1] = F.a1 * F.s0; W[0][2] = F.a1 * F.r13; W[0][3] = F.a1 * F.r14;
  W[1][0] = F.a2; W[1][1] = F.a2 * F.s1; W[1][2] = F.a2 * F.r23; W[1][3] = F.a2 * F.r24;
  W[2][0] = T(0); W[2][1] = T(0);        W[2][2] = F.a3;         W[2][3] = T(0);
  W[3][0] = T(0); W[3][1] = T(0);        W[3][2] = T(0);         W[3][3] = F.a4;
}

template <int LIM, class T> __device__ __forceinline__ T limiter_phi(T theta) {
  if (LIM == L_NONE) return T(0);
  if (LIM == L_LW) return T(1);
  T a = T(0.5) * (T(1) + theta);
  T m = a < T(2) ? a : T(2);
  T b = T(2) * theta;
  m = m < b ? m : b;
  return m > T(0) ? m : T(0);
}

__device__ __forceinline__ double ratio(double a, double b) { return a / b; }
__device__ __forceinline__ float ratio(float a, float b) { return __fdividef(a, b); }

// Fluctuations (eqs. fluc:m, fluc:p) and limited correction flux (eq.
// limiter) of face I, with its left and right neighbour faces for the upwind
// ratio theta (full four-component dot products).  The waves W[p][k] = a_p
// r_p have structural zeros (families 3 and 4 carry one component each, the
// acoustic families all four); the sums below leave out the products with
// those zeros, which changes no value (x + 0 = x, and the binary64 order of
// the remaining terms is that of the full sums), and each family reads only
// its own wave of the upwind face.
template <int LIM, class T>
__device__ __forceinline__ T coef_of(T s, T wdotw, T wup, T lam) {
  T theta = wdotw > T(0) ? ratio(wup, wdotw) : T(0);
  T phi = wdotw > T(0) ? limiter_phi<LIM, T>(theta) : T(0);
  T as = fabs(s);
  return as * (T(1) - lam * as) * phi;
}
template <int LIM, class T>
__device__ __forceinline__ void flux4(const Face4<T> &I, const Face4<T> &Lf, const Face4<T> &Rf,
                                      T lam, T am[4], T ap[4], T F[4]) {
  // waves of this face, acoustic families 0 and 1
  const T W00 = I.a1, W01 = I.a1 * I.s0, W02 = I.a1 * I.r13, W03 = I.a1 * I.r14;
  const T W10 = I.a2, W11 = I.a2 * I.s1, W12 = I.a2 * I.r23, W13 = I.a2 * I.r24;
  const T s0 = I.s0, s1 = I.s1, u = I.u;
  const T sm0 = s0 < T(0) ? s0 : T(0), sp0 = s0 > T(0) ? s0 : T(0);
  const T sm1 = s1 < T(0) ? s1 : T(0), sp1 = s1 > T(0) ? s1 : T(0);
  const T smu = u < T(0) ? u : T(0), spu = u > T(0) ? u : T(0);
  // sum over the families in the order 0, 1, 2, 3 of s^- W (s^+ W)
  am[0] = (T(0) + sm0 * W00) + sm1 * W10;
  ap[0] = (T(0) + sp0 * W00) + sp1 * W10;
  am[1] = (T(0) + sm0 * W01) + sm1 * W11;
  ap[1] = (T(0) + sp0 * W01) + sp1 * W11;
  am[2] = ((T(0) + sm0 * W02) + sm1 * W12) + smu * I.a3;
  ap[2] = ((T(0) + sp0 * W02) + sp1 * W12) + spu * I.a3;
  am[3] = ((T(0) + sm0 * W03) + sm1 * W13) + smu * I.a4;
  ap[3] = ((T(0) + sp0 * W03) + sp1 * W13) + spu * I.a4;
  // the upwind face's wave of each family (values selected, so that the
  // faces stay in registers)
  const bool l0 = s0 > T(0), l1 = s1 > T(0), lu = u > T(0);
  const T ua1 = l0 ? Lf.a1 : Rf.a1, us0 = l0 ? Lf.s0 : Rf.s0;
  const T ur13 = l0 ? Lf.r13 : Rf.r13, ur14 = l0 ? Lf.r14 : Rf.r14;
  const T ua2 = l1 ? Lf.a2 : Rf.a2, us1 = l1 ? Lf.s1 : Rf.s1;
  const T ur23 = l1 ? Lf.r23 : Rf.r23, ur24 = l1 ? Lf.r24 : Rf.r24;
  const T ua3 = lu ? Lf.a3 : Rf.a3, ua4 = lu ? Lf.a4 : Rf.a4;
  const T V00 = ua1, V01 = ua1 * us0, V02 = ua1 * ur13, V03 = ua1 * ur14;
  const T V10 = ua2, V11 = ua2 * us1, V12 = ua2 * ur23, V13 = ua2 * ur24;
  const T c0 = coef_of<LIM, T>(s0, (((T(0) + W00 * W00) + W01 * W01) + W02 * W02) + W03 * W03,
                               (((T(0) + V00 * W00) + V01 * W01) + V02 * W02) + V03 * W03, lam);
  const T c1 = coef_of<LIM, T>(s1, (((T(0) + W10 * W10) + W11 * W11) + W12 * W12) + W13 * W13,
                               (((T(0) + V10 * W10) + V11 * W11) + V12 * W12) + V13 * W13, lam);
  const T c2 = coef_of<LIM, T>(u, T(0) + I.a3 * I.a3, T(0) + ua3 * I.a3, lam);
  const T c3 = coef_of<LIM, T>(u, T(0) + I.a4 * I.a4, T(0) + ua4 * I.a4, lam);
  F[0] = T(0.5) * (c0 * W00 + c1 * W10);
  F[1] = T(0.5) * (c0 * W01 + c1 * W11);
  F[2] = T(0.5) * ((c0 * W02 + c1 * W12) + c2 * I.a3);
  F[3] = T(0.5) * ((c0 * W03 + c1 * W13) + c3 * I.a4);
}

// Cell update of eq. fv-hr.  binary64 as written; binary32 with COMP: the
// old value and the two increments summed with error-free two-sums and
// rounded once.
template <bool COMP>
__device__ __forceinline__ double update(double q, double am_r, double ap_l, double F_r, double F_l,
                                         double lam) {
  return q - lam * (am_r + ap_l) - lam * (F_r - F_l);
}
__device__ __forceinline__ void two_sum3(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
template <bool COMP>
__device__ __forceinline__ float update(float q, float am_r, float ap_l, float F_r, float F_l,
                                        float lam) {
  if (!COMP) return q - lam * (am_r + ap_l) - lam * (F_r - F_l);
  float t1 = -lam * (am_r + ap_l);
  float t2 = -lam * (F_r - F_l);
  float s, e1, e2;
  two_sum3(q, t1, s, e1);
  two_sum3(s, t2, s, e2);
  return s + (e1 + e2);
}

// |s| as an orderable bit pattern (NaN above every number)
__device__ __forceinline__ unsigned long long speed_bits(double s) {
  return (unsigned long long)__double_as_longlong(s) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long speed_bits(float s) {
  float a = fabsf(s);
  if (a != a) return 0x7ff8000000000000ull;
  return speed_bits((double)a);
}
// Running max |s| of a march in the precision's own bits (binary32: 32-bit
// patterns, every NaN above +inf), widened to the binary64 pattern of the
// domain scalars once per march.
template <class T> struct Speed;
template <> struct Speed<double> {
  typedef unsigned long long B;
  __device__ static B bits(double s) { return speed_bits(s); }
  __device__ static unsigned long long wide(B b) { return b; }
};
template <> struct Speed<float> {
  typedef unsigned B;
  __device__ static B bits(float s) { return __float_as_uint(fabsf(s)); }
  __device__ static unsigned long long wide(B b) {
    return b > 0x7f800000u ? 0x7ff8000000000000ull : speed_bits((double)__uint_as_float(b));
  }
};

// ---------------------------------------------------------------------------
// Line march: extended cells j = 0, 1, ... (two ghost cells, the line's
// cells, two ghost cells) are pushed in order; face j lies between cells j-1
// and j.  From j = 4 on, a push returns the update of cell j-2.  gl(j) = the
// line coordinate of the left cell of face j decides what the statistics see:
// max |s| over the faces of the domain cells, the non-real test over every
// face of the extended line (as the reference evaluation does).
// ---------------------------------------------------------------------------
template <class T, int LIM, bool COMP> struct March4 {
  T beta, lam;
  T c1[4], c2[4], z1[3];
  Face4<T> fm1, fm2;
  T apl[4], Fl[4];
  typename Speed<T>::B smax;
  bool nonreal;

  __device__ __forceinline__ void init(T b, T l) {
    beta = b;
    lam = l;
    smax = 0;
    nonreal = false;
  }
  // n = domain cells along the line; gl = line coordinate of the left cell of
  // face j; valid = this lane's line exists
  __device__ __forceinline__ bool push(int j, const T q[4], T out[4], int gl, int n, bool valid) {
    T r = inv_q1(q[0]);
    T z[3] = {q[1] * r, q[2] * r, q[3] * r};
    bool done = false;
    if (j > 0) {
      Face4<T> f;
      bool nr = roe4(beta, c1, z1, q, z, f);
      if (valid && gl >= -2 && gl <= n) nonreal |= nr;
      if (valid && gl >= -1 && gl <= n - 1) {
        typename Speed<T>::B b0 = Speed<T>::bits(f.s0), b1 = Speed<T>::bits(f.s1),
            b2 = Speed<T>::bits(f.u);
        smax = b0 > smax ? b0 : smax;
        smax = b1 > smax ? b1 : smax;
        smax = b2 > smax ? b2 : smax;
      }
      if (j >= 3) {
        T am[4], ap[4], F[4];
        flux4<LIM, T>(fm1, fm2, f, lam, am, ap, F);
        if (j >= 4) {
#pragma unroll
          for (int k = 0; k < 4; k++) out[k] = update<COMP>(c2[k], am[k], apl[k], F[k], Fl[k], lam);
          done = true;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
          apl[k] = ap[k];
          Fl[k] = F[k];
        }
      }
      fm2 = fm1;
      fm1 = f;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      c2[k] = c1[k];
      c1[k] = q[k];
    }
    z1[0] = z[0]; z1[1] = z[1]; z1[2] = z[2];
    return done;
  }
  // push of a cell j >= 4 (no start-up cases, so that consecutive cells can
  // be interleaved): the same operations as push, returning the update of
  // cell j - 2
  __device__ __forceinline__ void step(const T q[4], T out[4], int gl, int n, bool valid) {
    T r = inv_q1(q[0]);
    T z[3] = {q[1] * r, q[2] * r, q[3] * r};
    Face4<T> f;
    bool nr = roe4(beta, c1, z1, q, z, f);
    if (valid && gl >= -2 && gl <= n) nonreal |= nr;
    if (valid && gl >= -1 && gl <= n - 1) {
      typename Speed<T>::B b0 = Speed<T>::bits(f.s0), b1 = Speed<T>::bits(f.s1),
          b2 = Speed<T>::bits(f.u);
      smax = b0 > smax ? b0 : smax;
      smax = b1 > smax ? b1 : smax;
      smax = b2 > smax ? b2 : smax;
    }
    T am[4], ap[4], F[4];
    flux4<LIM, T>(fm1, fm2, f, lam, am, ap, F);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      out[k] = update<COMP>(c2[k], am[k], apl[k], F[k], Fl[k], lam);
      apl[k] = ap[k];
      Fl[k] = F[k];
    }
    fm2 = fm1;
    fm1 = f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      c2[k] = c1[k];
      c1[k] = q[k];
    }
    z1[0] = z[0]; z1[1] = z[1]; z1[2] = z[2];
  }
};

// warp-wide statistics of a march into the scalars
__device__ __forceinline__ void flush_stats(Scal3 *S, unsigned long long smax, bool nonreal) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_xor_sync(0xffffffffu, smax, o);
    smax = v > smax ? v : smax;
  }
  bool nr = __any_sync(0xffffffffu, nonreal);
  if ((threadIdx.x & 31) == 0) {
    if (smax) atomicMax(&S->smax_bits, smax);
    if (nr) atomicOr(&S->status_bits, S_NONREAL);
  }
}

// field order of each sweep: normal momentum second
__device__ __forceinline__ int perm(int dir, int k) {
  // x1: (0,1,2,3); x2: (0,2,1,3); x3: (0,3,1,2)
  return dir == 0 ? k : dir == 1 ? (k == 1 ? 2 : k == 2 ? 1 : k) : (k == 0 ? 0 : k == 1 ? 3 : k - 1);
}

// ---------------------------------------------------------------------------
// x1 sweep: a warp takes a segment of one row, 64 cells, lane l holding
// cells x0 - 2 + 2l and x0 - 1 + 2l; each lane computes the faces on the
// left of its two cells, the neighbour faces and cells come from the
// adjacent lanes by shuffles, lanes 1..30 update and store cells x0 ..
// x0 + 59.  Coalesced two-element loads and stores, no shared memory.
// ---------------------------------------------------------------------------
constexpr int X3_OUT = 60;

template <class T> __device__ __forceinline__ T shfl_up1(T v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}
template <class T> __device__ __forceinline__ T shfl_dn1(T v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}
// a neighbour's face: every field the upwind waves use
template <class T> __device__ __forceinline__ Face4<T> face_up(const Face4<T> &F) {
  Face4<T> o;
  o.s0 = shfl_up1(F.s0); o.s1 = shfl_up1(F.s1); o.u = shfl_up1(F.u);
  o.a1 = shfl_up1(F.a1); o.a2 = shfl_up1(F.a2); o.a3 = shfl_up1(F.a3); o.a4 = shfl_up1(F.a4);
  o.r13 = shfl_up1(F.r13); o.r23 = shfl_up1(F.r23); o.r14 = shfl_up1(F.r14);
  o.r24 = shfl_up1(F.r24);
  return o;
}
template <class T> __device__ __forceinline__ Face4<T> face_dn(const Face4<T> &F) {
  Face4<T> o;
  o.s0 = shfl_dn1(F.s0); o.s1 = shfl_dn1(F.s1); o.u = shfl_dn1(F.u);
  o.a1 = shfl_dn1(F.a1); o.a2 = shfl_dn1(F.a2); o.a3 = shfl_dn1(F.a3); o.a4 = shfl_dn1(F.a4);
  o.r13 = shfl_dn1(F.r13); o.r23 = shfl_dn1(F.r23); o.r14 = shfl_dn1(F.r14);
  o.r24 = shfl_dn1(F.r24);
  return o;
}

template <class T> struct Pair2;
template <> struct Pair2<double> { typedef double2 V; };
template <> struct Pair2<float> { typedef float2 V; };

template <class T, int LIM, bool COMP>
__global__ void __launch_bounds__(128) k3_sweep_x(Args3 A) {
  Scal3 *S = A.S;
  if (S->done) return;
  typedef typename Pair2<T>::V V2;
  const Dom3 &D = A.d;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nx = D.nx;
  const long long nrows = (long long)D.ny * D.nz;
  const int segs = (nx + X3_OUT - 1) / X3_OUT;
  const long long items = nrows * segs;
  const T lam = sizeof(T) == 8 ? (T)S->lam : (T)S->lam32;
  const T beta = (T)A.beta;
  const T *in[4] = {(const T *)A.in[0], (const T *)A.in[1], (const T *)A.in[2],
                    (const T *)A.in[3]};
  T *out[4] = {(T *)A.out[0], (T *)A.out[1], (T *)A.out[2], (T *)A.out[3]};
  typename Speed<T>::B smax = 0;
  bool nonreal = false;
  for (long long t = warp; t < items; t += nwarps) {
    const long long row = t / segs;
    const int x0 = (int)(t - row * segs) * X3_OUT;
    const int ca = x0 - 2 + 2 * lane;
    const long long rb = row * D.pitch;
    T qa[4], qb[4];
    if (x0 >= 2 && x0 + X3_OUT + 2 <= nx) {
#pragma unroll
      for (int f = 0; f < 4; f++) {
        V2 v = *(const V2 *)(in[f] + rb + ca);
        qa[f] = v.x;
        qb[f] = v.y;
      }
    } else {
      bool fa, fb;
      const int ia = map_cell(ca, nx, D.bc[0], D.bc[1], fa);
      const int ib = map_cell(ca + 1, nx, D.bc[0], D.bc[1], fb);
#pragma unroll
      for (int f = 0; f < 4; f++) {
        qa[f] = in[f][rb + ia];
        qb[f] = in[f][rb + ib];
      }
      if (fa) qa[1] = -qa[1];
      if (fb) qb[1] = -qb[1];
    }
    T ra = inv_q1(qa[0]), rbq = inv_q1(qb[0]);
    T za[3] = {qa[1] * ra, qa[2] * ra, qa[3] * ra};
    T zb[3] = {qb[1] * rbq, qb[2] * rbq, qb[3] * rbq};
    T ql[4], zl[3];
#pragma unroll
    for (int f = 0; f < 4; f++) ql[f] = shfl_up1(qb[f]);
#pragma unroll
    for (int f = 0; f < 3; f++) zl[f] = shfl_up1(zb[f]);
    Face4<T> FA, FB;
    bool nrA = roe4(beta, ql, zl, qa, za, FA);
    bool nrB = roe4(beta, qa, za, qb, zb, FB);
    // statistics: face A of lane 0 has no left cell; |s| over the faces of
    // the domain cells, the non-real test over the extended line's
    const int glA = ca - 1, glB = ca;
    if (lane > 0) {
      if (glA >= -2 && glA <= nx) nonreal |= nrA;
      if (glA >= -1 && glA <= nx - 1) {
        typename Speed<T>::B b0 = Speed<T>::bits(FA.s0), b1 = Speed<T>::bits(FA.s1),
                             b2 = Speed<T>::bits(FA.u);
        smax = b0 > smax ? b0 : smax; smax = b1 > smax ? b1 : smax; smax = b2 > smax ? b2 : smax;
      }
    }
    if (glB >= -2 && glB <= nx) nonreal |= nrB;
    if (glB >= -1 && glB <= nx - 1) {
      typename Speed<T>::B b0 = Speed<T>::bits(FB.s0), b1 = Speed<T>::bits(FB.s1),
                           b2 = Speed<T>::bits(FB.u);
      smax = b0 > smax ? b0 : smax; smax = b1 > smax ? b1 : smax; smax = b2 > smax ? b2 : smax;
    }
    const Face4<T> LB = face_up(FB), RA = face_dn(FA);
    T amA[4], apA[4], FFA[4], amB[4], apB[4], FFB[4];
    flux4<LIM, T>(FA, LB, FB, lam, amA, apA, FFA);
    flux4<LIM, T>(FB, FA, RA, lam, amB, apB, FFB);
    T amN[4], FFN[4];      // the next lane's face A: the right face of cell ca + 1
#pragma unroll
    for (int f = 0; f < 4; f++) {
      amN[f] = shfl_dn1(amA[f]);
      FFN[f] = shfl_dn1(FFA[f]);
    }
    if (lane >= 1 && lane <= 30) {
      T na[4], nb[4];
#pragma unroll
      for (int f = 0; f < 4; f++) {
        na[f] = update<COMP>(qa[f], amB[f], apA[f], FFB[f], FFA[f], lam);
        nb[f] = update<COMP>(qb[f], amN[f], apB[f], FFN[f], FFB[f], lam);
      }
      if (ca + 1 < nx) {
#pragma unroll
        for (int f = 0; f < 4; f++) {
          V2 v;
          v.x = na[f];
          v.y = nb[f];
          *(V2 *)(out[f] + rb + ca) = v;
        }
      } else if (ca < nx) {
#pragma unroll
        for (int f = 0; f < 4; f++) out[f][rb + ca] = na[f];
      }
    }
  }
  flush_stats(S, Speed<T>::wide(smax), nonreal);
}

// ---------------------------------------------------------------------------
// x2 / x3 sweep: lanes on 32 consecutive x1 columns, marching along x2 or x3
// ---------------------------------------------------------------------------
template <class T, int LIM, bool COMP>
__global__ void __launch_bounds__(128) k3_sweep_v(Args3 A) {
  Scal3 *S = A.S;
  if (S->done) return;
  const Dom3 &D = A.d;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int dir = A.dir;
  const int n = dir == 1 ? D.ny : D.nz;               // cells along the march
  const int no = dir == 1 ? D.nz : D.ny;              // the other transverse extent
  const long long stride = dir == 1 ? (long long)D.pitch : (long long)D.pitch * D.ny;
  const long long ostride = dir == 1 ? (long long)D.pitch * D.ny : (long long)D.pitch;
  const int bclo = D.bc[2 * dir], bchi = D.bc[2 * dir + 1];
  const int TY = A.tile;
  const int tx = (D.nx + 31) / 32, ty = (n + TY - 1) / TY;
  const long long tiles = (long long)tx * ty * no;
  const T lam = sizeof(T) == 8 ? (T)S->lam : (T)S->lam32;
  int pf[4];
  for (int k = 0; k < 4; k++) pf[k] = perm(dir, k);
  const T *in[4] = {(const T *)A.in[pf[0]], (const T *)A.in[pf[1]], (const T *)A.in[pf[2]],
                    (const T *)A.in[pf[3]]};
  T *out[4] = {(T *)A.out[pf[0]], (T *)A.out[pf[1]], (T *)A.out[pf[2]], (T *)A.out[pf[3]]};
  typename Speed<T>::B smax = 0;
  bool nonreal = false;
  for (long long t = warp; t < tiles; t += nwarps) {
    const int xt = (int)(t % tx);
    const long long rest = t / tx;
    const int yt = (int)(rest % ty);
    const int o = (int)(rest / ty);
    const int x = xt * 32 + lane;
    const bool valid = x < D.nx;
    const int xc = valid ? x : D.nx - 1;
    const long long base = (long long)o * ostride + xc;
    const int g0 = yt * TY;
    const int len = min(TY, n - g0) + 4;
    March4<T, LIM, COMP> m;
    m.init((T)A.beta, lam);
    // a tile whose marched cells (two halo cells at each end) all lie inside
    // the line reads them without the border rules
    const bool inner = g0 >= 2 && g0 + len - 3 <= n - 1;
    auto load = [&](int j, T q[4]) {
      bool flip = false;
      const int c = inner ? g0 - 2 + j : map_cell(g0 - 2 + j, n, bclo, bchi, flip);
      const long long off = base + (long long)c * stride;
#pragma unroll
      for (int k = 0; k < 4; k++) q[k] = in[k][off];
      if (flip) q[1] = -q[1];
    };
    T nxt[4];
    load(0, nxt);
    // start-up: cells 0..3 (no update yet); len >= 5
    for (int j = 0; j < 4; j++) {
      T q[4] = {nxt[0], nxt[1], nxt[2], nxt[3]};
      load(j + 1, nxt);
      T ov[4];
      m.push(j, q, ov, g0 - 3 + j, n, valid);
    }
#pragma unroll 2
    for (int j = 4; j < len; j++) {
      T q[4] = {nxt[0], nxt[1], nxt[2], nxt[3]};
      if (j + 1 < len) load(j + 1, nxt);
      T ov[4];
      m.step(q, ov, g0 - 3 + j, n, valid);
      if (valid) {
        long long off = base + (long long)(g0 + j - 4) * stride;
#pragma unroll
        for (int k = 0; k < 4; k++) out[k][off] = ov[k];
      }
    }
    smax = m.smax > smax ? m.smax : smax;
    nonreal |= m.nonreal;
  }
  flush_stats(S, Speed<T>::wide(smax), nonreal);
}

// ---------------------------------------------------------------------------
// Source: forward Euler with the 7-point Laplacian of z = (q2, q3, q4)/q1,
// summed as ((W + E) + (S + N) - 4 C) + ((B + T) - 2 C).
// ---------------------------------------------------------------------------
// state of cell (i, j, k), ghost cells by the border rules (the normal
// momentum of a mirrored cell negated), and its velocity z = (q2, q3, q4)/q1
template <class T>
__device__ __forceinline__ void qat(const Args3 &A, int i, int j, int k, T q[4]) {
  const Dom3 &D = A.d;
  bool fx = false, fy = false, fz = false;
  int ci = map_cell(i, D.nx, D.bc[0], D.bc[1], fx);
  int cj = map_cell(j, D.ny, D.bc[2], D.bc[3], fy);
  int ck = map_cell(k, D.nz, D.bc[4], D.bc[5], fz);
  long long off = ((long long)ck * D.ny + cj) * D.pitch + ci;
  const T *const *in = (const T *const *)A.in;
#pragma unroll
  for (int f = 0; f < 4; f++) q[f] = in[f][off];
  if (fx) q[1] = -q[1];
  if (fy) q[2] = -q[2];
  if (fz) q[3] = -q[3];
}
template <class T> __device__ __forceinline__ void zof3(const T q[4], T z[3]) {
  T r = inv_q1(q[0]);
  z[0] = q[1] * r;
  z[1] = q[2] * r;
  z[2] = q[3] * r;
}

// One block marches a tile of SRC3_TX x SRC3_TY cells of the (x1, x2) plane
// along x3 through a chunk of SRC3_KCH planes.  Every cell's velocity z is
// formed once per plane: the tile's cells and a one-cell ring around it go
// to shared memory for the x1 and x2 neighbours (the ring's cells are the
// border rules' ghosts where the tile meets a border), and each thread keeps
// the z of planes k-1, k and k+1 of its own cell in registers.  The state a
// thread needs next (its own cell two planes ahead, its ring cell one plane
// ahead) is loaded while the current plane is formed.  Threads of a tile
// that overhangs the domain form ghost or clamped cells and store nothing.
constexpr int SRC3_TX = 32, SRC3_TY = 8, SRC3_KCH = 16;
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k3_source(Args3 A) {
  Scal3 *S = A.S;
  if (S->done) return;
  const Dom3 &D = A.d;
  __shared__ T sz[3][SRC3_TY + 2][SRC3_TX + 2];
  const int tx = threadIdx.x % SRC3_TX, ty = threadIdx.x / SRC3_TX;
  const T coef = sizeof(T) == 8 ? (T)S->coef : (T)S->coef32;
  T *const *out = (T *const *)A.out;
  // the ring cell this thread forms (threads 0 .. 2 (TX + TY) - 1): the
  // x1-low and x1-high columns, then the x2-low and x2-high rows
  const int h = threadIdx.x;
  int hx = -1, hy = -1;
  if (h < SRC3_TY) { hx = 0; hy = 1 + h; }
  else if (h < 2 * SRC3_TY) { hx = SRC3_TX + 1; hy = 1 + h - SRC3_TY; }
  else if (h < 2 * SRC3_TY + SRC3_TX) { hx = 1 + h - 2 * SRC3_TY; hy = 0; }
  else if (h < 2 * SRC3_TY + 2 * SRC3_TX) { hx = 1 + h - 2 * SRC3_TY - SRC3_TX; hy = SRC3_TY + 1; }
  const int ntj = (D.ny + SRC3_TY - 1) / SRC3_TY, nkc = (D.nz + SRC3_KCH - 1) / SRC3_KCH;
  const int i0 = blockIdx.x * SRC3_TX, i = i0 + tx;
  for (int jt = blockIdx.y; jt < ntj; jt += gridDim.y) {
    const int j0 = jt * SRC3_TY, j = j0 + ty;
    const bool own = i < D.nx && j < D.ny;
    const int hi = i0 - 1 + hx, hj = j0 - 1 + hy;
    for (int kc = blockIdx.z; kc < nkc; kc += gridDim.z) {
      const int k0 = kc * SRC3_KCH, k1 = min(D.nz, k0 + SRC3_KCH);
      T zb[3], zc[3], zt[3], qc[4], qt[4], hq[4];
      qat<T>(A, i, j, k0 - 1, qc);
      zof3<T>(qc, zb);
      qat<T>(A, i, j, k0, qc);
      zof3<T>(qc, zc);
      qat<T>(A, i, j, k0 + 1, qt);
      if (hx >= 0) qat<T>(A, hi, hj, k0, hq);
      for (int k = k0; k < k1; k++) {
        T qn[4];
        if (k + 1 < k1) qat<T>(A, i, j, k + 2, qn);
        zof3<T>(qt, zt);
#pragma unroll
        for (int f = 0; f < 3; f++) sz[f][ty + 1][tx + 1] = zc[f];
        if (hx >= 0) {
          T zh[3];
          zof3<T>(hq, zh);
#pragma unroll
          for (int f = 0; f < 3; f++) sz[f][hy][hx] = zh[f];
          if (k + 1 < k1) qat<T>(A, hi, hj, k + 1, hq);
        }
        __syncthreads();
        if (own) {
          const long long off = ((long long)k * D.ny + j) * D.pitch + i;
          out[0][off] = qc[0];
#pragma unroll
          for (int f = 0; f < 3; f++) {
            T L = ((sz[f][ty + 1][tx] + sz[f][ty + 1][tx + 2]) +
                   (sz[f][ty][tx + 1] + sz[f][ty + 2][tx + 1]) - T(4) * zc[f]) +
                  ((zb[f] + zt[f]) - T(2) * zc[f]);
            out[1 + f][off] = qc[1 + f] + coef * L;
          }
        }
        __syncthreads();
#pragma unroll
        for (int f = 0; f < 3; f++) {
          zb[f] = zc[f];
          zc[f] = zt[f];
        }
#pragma unroll
        for (int f = 0; f < 4; f++) {
          qc[f] = qt[f];
          if (k + 1 < k1) qt[f] = qn[f];
        }
      }
    }
  }
}

// plain copy of the four planes (a step whose enabled sub-steps end in the
// swept planes)
template <class T> __global__ void k3_copy(Args3 A) {
  if (A.S->done) return;
  const Dom3 &D = A.d;
  const long long n = D.plane;
  for (int f = 0; f < 4; f++) {
    const T *src = (const T *)A.in[f];
    T *dst = (T *)A.out[f];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
      dst[c] = src[c];
  }
}

// speed-only pass over every face of the domain cells, all three directions
template <class T> __global__ void k3_speeds(Args3 A) {
  const Dom3 &D = A.d;
  const long long nf[3] = {(long long)(D.nx + 1) * D.ny * D.nz, (long long)D.nx * (D.ny + 1) * D.nz,
                           (long long)D.nx * D.ny * (D.nz + 1)};
  const T *const *in = (const T *const *)A.in;
  unsigned long long smax = 0ull;
  bool nonreal = false;
  for (int dir = 0; dir < 3; dir++) {
    const int n = dir == 0 ? D.nx : dir == 1 ? D.ny : D.nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nf[dir];
         e += (long long)gridDim.x * blockDim.x) {
      int i, j, k, a;
      if (dir == 0) {
        a = (int)(e % (D.nx + 1)); long long r = e / (D.nx + 1);
        j = (int)(r % D.ny); k = (int)(r / D.ny); i = a;
      } else if (dir == 1) {
        i = (int)(e % D.nx); long long r = e / D.nx;
        a = (int)(r % (D.ny + 1)); k = (int)(r / (D.ny + 1)); j = a;
      } else {
        i = (int)(e % D.nx); long long r = e / D.nx;
        j = (int)(r % D.ny); a = (int)(r / D.ny); k = a;
      }
      T cell[2][4], z[2][3];
      for (int s = 0; s < 2; s++) {
        int ii = i, jj = j, kk = k;
        if (dir == 0) ii = a - 1 + s; else if (dir == 1) jj = a - 1 + s; else kk = a - 1 + s;
        bool fl;
        int g = dir == 0 ? ii : dir == 1 ? jj : kk;
        int cg = map_cell(g, n, D.bc[2 * dir], D.bc[2 * dir + 1], fl);
        if (dir == 0) ii = cg; else if (dir == 1) jj = cg; else kk = cg;
        long long off = ((long long)kk * D.ny + jj) * D.pitch + ii;
        for (int f = 0; f < 4; f++) cell[s][f] = in[perm(dir, f)][off];
        if (fl) cell[s][1] = -cell[s][1];
        T r = inv_q1(cell[s][0]);
        for (int f = 0; f < 3; f++) z[s][f] = cell[s][1 + f] * r;
      }
      Face4<T> F;
      nonreal |= roe4((T)A.beta, cell[0], z[0], cell[1], z[1], F);
      unsigned long long b0 = speed_bits(F.s0), b1 = speed_bits(F.s1), b2 = speed_bits(F.u);
      smax = b0 > smax ? b0 : smax;
      smax = b1 > smax ? b1 : smax;
      smax = b2 > smax ? b2 : smax;
    }
  }
  flush_stats(A.S, smax, nonreal);
}

// ---------------------------------------------------------------------------
// Step bookkeeping (binary64 for both precisions), section 4's CFL rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_scalars3(Scal3 *S, const Args3 &A) {
  S->lam = __ddiv_rn(S->dt, A.dx);
  S->coef = __ddiv_rn(__dmul_rn(S->dt, A.delta), __dmul_rn(A.dx, A.dx));
  S->lam32 = (float)S->lam;
  S->coef32 = (float)S->coef;
}

// host-side import / export of binary64 total variables (layout of fvna.h:
// field f, cell (i, j, k) at f*n + (k*ny + j)*nx + i)
template <class T> __global__ void k3_import(Args3 A, const double *q) {
  const Dom3 &D = A.d;
  const long long n = (long long)D.nx * D.ny * D.nz;
  T *const *out = (T *const *)A.out;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    long long row = c / D.nx;
    long long off = row * D.pitch + (c - row * D.nx);
    for (int f = 0; f < 4; f++) {
      double v = q[f * n + c];
      out[f][off] = (T)(f == 0 && sizeof(T) == 4 ? v - 1.0 : v);
    }
  }
}
// what: 0 the four fields, 1 p' = q1 - 1
template <class T> __global__ void k3_export(Args3 A, double *q, int what) {
  const Dom3 &D = A.d;
  const long long n = (long long)D.nx * D.ny * D.nz;
  const T *const *in = (const T *const *)A.in;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    long long row = c / D.nx;
    long long off = row * D.pitch + (c - row * D.nx);
    double a = (double)in[0][off];
    if (what == 1) {
      q[c] = sizeof(T) == 4 ? a : a - 1.0;
      continue;
    }
    q[c] = sizeof(T) == 4 ? a + 1.0 : a;
    for (int f = 1; f < 4; f++) q[f * n + c] = (double)in[f][off];
  }
}

}  // namespace d3
}  // namespace fvna
