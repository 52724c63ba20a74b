// fvna_device.cuh -- device code of the finite-volume step (arXiv 1311.3004,
// section 3): Roe solver, limited corrections, the line marcher shared by the
// two sweeps, border handling, and the sweep kernels.  Included by one
// translation unit per precision:
//   fvna_fp64.cu  (binary64, compiled with -fmad=false so that every product
//                  and sum rounds as written: the formulas below are evaluated
//                  in the same order as the paper's definitions are written),
//   fvna_fp32.cu  (binary32 perturbation variables, FMA allowed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fvna_types.h"

namespace fvna {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T dmin0(T s) { return s < T(0) ? s : T(0); }
template <class T> __device__ __forceinline__ T dmax0(T s) { return s > T(0) ? s : T(0); }

// max that lets a NaN through (a NaN speed must never be hidden)
__device__ __forceinline__ double max_nan(double a, double b) {
  if (a != a || b != b) return a != a ? a : b;
  return a > b ? a : b;
}

// atomic max of a non-negative double (or NaN) by its bit pattern: for such
// values the IEEE encoding orders like an unsigned integer, and every NaN
// with a clear sign bit sorts above +inf.
__device__ __forceinline__ void atomic_max_speed(unsigned long long *slot, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (v != v) b = 0x7ff8000000000000ull;
  atomicMax(slot, b);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = max_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_or(int v) {
  return __reduce_or_sync(0xffffffffu, (unsigned)v);
}

// ---------------------------------------------------------------------------
// Driven borders (section 4.1 eq. OurTaylorS, section 4.2 eq. hifuBC).
// Total-variable form, evaluated in the order of the definitions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void taylor_total(const DomDev &D, double x, double y, double t,
                                             double out[3]) {
  double q1 = 1.0 - D.taylor_ratio * tanh(x * D.taylor_ct + y * D.taylor_st - t);
  out[0] = q1;
  out[1] = (q1 - 1.0) * D.taylor_ct;
  out[2] = (q1 - 1.0) * D.taylor_st;
}

__device__ __forceinline__ double hifu_envelope(int kind, double tau) {
  double w = tau * 0.25;
  double w2 = w * w;
  double w4 = w2 * w2;
  double w8 = w4 * w4;
  double w10 = w8 * w2;
  if (kind == 0) {
    if (tau <= 0.0) return 0.0;
    return exp(-1.0 / w10);
  }
  return exp(-w10);
}

// g of eq. hifuBC with tau = t + x2^2/(2F) - x1 (x1 <= 0 at a ghost centre)
__device__ __forceinline__ double hifu_g(const DomDev &D, double x1, double x2, double t) {
  const double two_pi = 6.283185307179586;
  double tau = t + x2 * x2 / (2.0 * D.focal) - x1;
  return D.amp * sin(two_pi * tau) * hifu_envelope(D.env, tau);
}

__device__ __forceinline__ void hifu_total(const DomDev &D, double x1, double x2, double t,
                                           double out[3]) {
  double g = hifu_g(D, x1, x2, t);
  double rn = sqrt(x2 * x2 + D.focal * D.focal);
  out[0] = 1.0 + g;
  out[1] = D.focal * g / rn;
  out[2] = -x2 * g / rn;
}

// ---------------------------------------------------------------------------
// Precision policies.  A cell is (a, b, c) = (q1 or q1-1, normal momentum,
// transverse momentum); the x2 sweep passes (q1, q3, q2).
// ---------------------------------------------------------------------------
struct P64 {
  typedef double T;
  static constexpr bool pert = false;
  // 1/q1 of a stored cell
  __device__ static __forceinline__ double rq1(double a) { return 1.0 / a; }
  __device__ static __forceinline__ double stored_q1(double q1) { return q1; }
  // driven value converted to the stored form
  __device__ static __forceinline__ void taylor(const DomDev &D, double x, double y, double t,
                                                double o[3]) { taylor_total(D, x, y, t, o); }
  __device__ static __forceinline__ void hifu(const DomDev &D, double x, double y, double t,
                                              double o[3]) { hifu_total(D, x, y, t, o); }
};

struct P32 {
  typedef float T;
  static constexpr bool pert = true;
  __device__ static __forceinline__ float rq1(float a) { return 1.0f / (1.0f + a); }
  // perturbation values computed directly (no 1 + small - 1 round trip)
  __device__ static __forceinline__ void taylor(const DomDev &D, double x, double y, double t,
                                                double o[3]) {
    double w = -D.taylor_ratio * tanh(x * D.taylor_ct + y * D.taylor_st - t);
    o[0] = w;
    o[1] = w * D.taylor_ct;
    o[2] = w * D.taylor_st;
  }
  __device__ static __forceinline__ void hifu(const DomDev &D, double x, double y, double t,
                                              double o[3]) {
    double g = hifu_g(D, x, y, t);
    double rn = sqrt(y * y + D.focal * D.focal);
    o[0] = g;
    o[1] = D.focal * g / rn;
    o[2] = -y * g / rn;
  }
};

// One interface: speeds and waves (family p: W[p][0..2]; family 3 has only a
// transverse component, kept in W2).
template <class T> struct Iface {
  T s0, s1, s2;
  T W0[3], W1[3];
  T W2;
};

// Roe solver of section 3.2 in binary64.  zb, zc are the per-cell z = q/q1.
// Returns true when the radicand of eqs. lambda1/lambda2 is negative.
__device__ __forceinline__ bool roe(const P64 &, double beta2, double aL, double bL, double cL,
                                    double zbL, double zcL, double aR, double bR, double cR,
                                    double zbR, double zcR, Iface<double> &I) {
  double Z1 = 0.5 * (aL + aR);
  double Z2 = 0.5 * (zbL + zbR);
  double Z3 = 0.5 * (zcL + zcR);
  double Phi = 1.0 + beta2 * (Z1 - 1.0);
  double rZ1 = 1.0 / Z1;
  double u = Z2 * rZ1;
  double v = Z3 * rZ1;
  double D = u * u - 2.0 * Z2 * u + Phi;
  bool nonreal = D < 0.0;
  double c = sqrt(D);
  I.s0 = u + c;
  I.s1 = u - c;
  I.s2 = u;
  double rc = 1.0 / c;
  double h = 0.5 * rc;
  double d1 = aR - aL;
  double d2 = bR - bL;
  double d3 = cR - cL;
  double r13 = v * (I.s0 - 2.0 * Z2) * rc;
  double r23 = v * (2.0 * Z2 - I.s1) * rc;
  double a1 = (d2 - I.s1 * d1) * h;
  double a2 = (I.s0 * d1 - d2) * h;
  double a3 = d3 - a1 * r13 - a2 * r23;
  I.W0[0] = a1; I.W0[1] = a1 * I.s0; I.W0[2] = a1 * r13;
  I.W1[0] = a2; I.W1[1] = a2 * I.s1; I.W1[2] = a2 * r23;
  I.W2 = a3;
  return nonreal;
}

// The same solver on perturbation variables in binary32: every 1 + small is
// carried as small (Z1 - 1, D - 1, c - 1), so the ambient state never cancels.
__device__ __forceinline__ bool roe(const P32 &, float beta2, float aL, float bL, float cL,
                                    float zbL, float zcL, float aR, float bR, float cR,
                                    float zbR, float zcR, Iface<float> &I) {
  float Z1p = 0.5f * (aL + aR);                 // Z1 - 1
  float Z2 = 0.5f * (zbL + zbR);
  float Z3 = 0.5f * (zcL + zcR);
  float rZ1 = 1.0f / (1.0f + Z1p);
  float u = Z2 * rZ1;
  float v = Z3 * rZ1;
  float dm = u * u - 2.0f * Z2 * u + beta2 * Z1p;  // D - 1
  bool nonreal = dm < -1.0f;
  float e = dm / (1.0f + sqrtf(1.0f + dm));     // sqrt(D) - 1
  float c = 1.0f + e;
  I.s0 = u + c;
  I.s1 = u - c;
  I.s2 = u;
  float rc = 1.0f / c;
  float h = 0.5f * rc;
  float d1 = aR - aL;
  float d2 = bR - bL;
  float d3 = cR - cL;
  float r13 = v * (I.s0 - 2.0f * Z2) * rc;
  float r23 = v * (2.0f * Z2 - I.s1) * rc;
  float a1 = (d2 - I.s1 * d1) * h;
  float a2 = (I.s0 * d1 - d2) * h;
  float a3 = d3 - a1 * r13 - a2 * r23;
  I.W0[0] = a1; I.W0[1] = a1 * I.s0; I.W0[2] = a1 * r13;
  I.W1[0] = a2; I.W1[1] = a2 * I.s1; I.W1[2] = a2 * r23;
  I.W2 = a3;
  return nonreal;
}

// Limiter function of eq. limiter for the ratio wup/wdotw; 0 when the wave is
// zero (wdotw = 0).  LIM is the limiter kind (MC, none = Godunov, LW).
template <class T> __device__ __forceinline__ T lim_ratio(T num, T den);
template <> __device__ __forceinline__ double lim_ratio<double>(double num, double den) {
  return num / den;
}
template <> __device__ __forceinline__ float lim_ratio<float>(float num, float den) {
  return __fdividef(num, den);
}

template <int LIM, class T> __device__ __forceinline__ T limited(T wup, T wdotw) {
  if (LIM == LIM_NONE) return T(0);
  if (LIM == LIM_LW) return wdotw > T(0) ? T(1) : T(0);
  T theta = lim_ratio<T>(wup, wdotw);
  T a = T(0.5) * (T(1) + theta);
  T m = a < T(2) ? a : T(2);
  T b = T(2) * theta;
  m = m < b ? m : b;
  m = m > T(0) ? m : T(0);
  return wdotw > T(0) ? m : T(0);
}

// Fluctuations (eqs. fluc:m, fluc:p) and the limited correction flux (eq.
// limiter) of interface I, with the waves of its left (Lf) and right (Rf)
// neighbours for the upwind ratio theta.
template <class T> struct FluxData {
  T am[3], ap[3], F[3];
};

template <int LIM, class T>
__device__ __forceinline__ T family_coef(T s, const T *W, const T *U, T lam) {
  T wdotw = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
  T wup = U[0] * W[0] + U[1] * W[1] + U[2] * W[2];
  T phi = limited<LIM, T>(wup, wdotw);
  T as = fabs(s);
  return as * (T(1) - lam * as) * phi;
}

template <int LIM, class T>
__device__ __forceinline__ void flux_data(const Iface<T> &I, const Iface<T> &Lf, const Iface<T> &Rf,
                                          T lam, FluxData<T> &o) {
  T coef0, coef1;
  const T sm2 = dmin0(I.s2), sp2 = dmax0(I.s2);
  if (I.s0 > T(0) && I.s1 < T(0)) {
    // subsonic interface (always the case for acoustic perturbations): the
    // first family moves right and the second left, so the sums over the
    // families reduce to one term each (the dropped terms are exact zeros)
    o.am[0] = I.s1 * I.W1[0];
    o.am[1] = I.s1 * I.W1[1];
    o.am[2] = I.s1 * I.W1[2] + sm2 * I.W2;
    o.ap[0] = I.s0 * I.W0[0];
    o.ap[1] = I.s0 * I.W0[1];
    o.ap[2] = I.s0 * I.W0[2] + sp2 * I.W2;
    coef0 = family_coef<LIM, T>(I.s0, I.W0, Lf.W0, lam);
    coef1 = family_coef<LIM, T>(I.s1, I.W1, Rf.W1, lam);
  } else {
    T sm0 = dmin0(I.s0), sm1 = dmin0(I.s1);
    T sp0 = dmax0(I.s0), sp1 = dmax0(I.s1);
#pragma unroll
    for (int k = 0; k < 2; k++) {
      T am = T(0), ap = T(0);
      am = am + sm0 * I.W0[k];
      ap = ap + sp0 * I.W0[k];
      am = am + sm1 * I.W1[k];
      ap = ap + sp1 * I.W1[k];
      o.am[k] = am;
      o.ap[k] = ap;
    }
    T am = T(0), ap = T(0);
    am = am + sm0 * I.W0[2];
    ap = ap + sp0 * I.W0[2];
    am = am + sm1 * I.W1[2];
    ap = ap + sp1 * I.W1[2];
    am = am + sm2 * I.W2;
    ap = ap + sp2 * I.W2;
    o.am[2] = am;
    o.ap[2] = ap;
    coef0 = family_coef<LIM, T>(I.s0, I.W0, I.s0 > T(0) ? Lf.W0 : Rf.W0, lam);
    coef1 = family_coef<LIM, T>(I.s1, I.W1, I.s1 > T(0) ? Lf.W1 : Rf.W1, lam);
  }
  T coef2;
  {
    T U = I.s2 > T(0) ? Lf.W2 : Rf.W2;
    T phi = limited<LIM, T>(U * I.W2, I.W2 * I.W2);
    T as = fabs(I.s2);
    coef2 = as * (T(1) - lam * as) * phi;
  }
  o.F[0] = T(0.5) * (coef0 * I.W0[0] + coef1 * I.W1[0]);
  o.F[1] = T(0.5) * (coef0 * I.W0[1] + coef1 * I.W1[1]);
  o.F[2] = T(0.5) * (coef0 * I.W0[2] + coef1 * I.W1[2] + coef2 * I.W2);
}

// Cell update of eq. fv-hr.  binary64: evaluated as written.
template <bool COMP>
__device__ __forceinline__ double cell_update(const P64 &, double q, double am_r, double ap_l,
                                              double F_r, double F_l, double lam) {
  return q - lam * (am_r + ap_l) - lam * (F_r - F_l);
}

// binary32 with COMP: the two increments of eq. fv-hr (fluctuations and the
// correction-flux difference) are added to the old value with error-free
// two-sums (Knuth) and their rounding errors folded back once (Neumaier), so
// the new value is rounded once from the exact sum of the two increments.
// Without COMP the update is evaluated as written.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
template <bool COMP>
__device__ __forceinline__ float cell_update(const P32 &, float q, float am_r, float ap_l,
                                             float F_r, float F_l, float lam) {
  if (!COMP) return q - lam * (am_r + ap_l) - lam * (F_r - F_l);
  float t1 = -lam * (am_r + ap_l);
  float t2 = -lam * (F_r - F_l);
  float s, e1, e2;
  two_sum(q, t1, s, e1);
  two_sum(s, t2, s, e2);
  return s + (e1 + e2);
}

// ---------------------------------------------------------------------------
// Line marcher: cells of one line are pushed in order; once four cells are
// in, every push updates the cell two behind (eq. fv-hr), using the
// interfaces on its two faces and their neighbours for the limiter.
// ---------------------------------------------------------------------------
template <class P> struct Marcher {
  typedef typename P::T T;
  T beta2, lam;
  int lim;
  // cells c-2, c-1 (old values) and z of c-1
  T a2_, b2_, c2_, a1_, b1_, c1_, zb1, zc1;
  Iface<T> Im2, Im1;          // interfaces c-2, c-1 (interface k lies between cells k-1, k)
  T ap_l[3], F_l[3];          // flux data of interface c-2 (left face of cell c-2)
  bool nonreal;

  __device__ __forceinline__ void first(T a, T b, T c) {
    T r = P::rq1(a);
    a1_ = a; b1_ = b; c1_ = c;
    zb1 = b * r; zc1 = c * r;
    nonreal = false;
  }
  // push cell 1..: compute the interface with the previous cell
  __device__ __forceinline__ void iface(T a, T b, T c, Iface<T> &I) {
    T r = P::rq1(a);
    T zb = b * r, zc = c * r;
    nonreal |= roe(P(), beta2, a1_, b1_, c1_, zb1, zc1, a, b, c, zb, zc, I);
    a2_ = a1_; b2_ = b1_; c2_ = c1_;
    a1_ = a; b1_ = b; c1_ = c;
    zb1 = zb; zc1 = zc;
  }
};

}  // namespace fvna
