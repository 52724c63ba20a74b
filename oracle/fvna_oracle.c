/*
 * fvna_oracle.c -- plain, slow FP64 CPU oracle of the finite-volume scheme of
 * Velasco-Segura & Rendon, "A Finite Volume Approach for the Simulation of
 * Nonlinear Dissipative Acoustic Wave Propagation" (arXiv 1311.3004).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the GPU library is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * What it computes (paper section 3, eqs. OurSysAdim, fs:cl1-fs:source,
 * fv-hr, fluc:m, fluc:p, limiter, the Roe matrix of section 3.2 and the CFL
 * rule at the start of section 4), written as plainly as possible:
 *
 *   state     q = (q1, q2, q3) = (rho/rho0)(1, u1/c0, u2/c0)      eq. adim:q
 *   flux      f_1 = (q2, (q2/q1)^2 + phi, q2 q3/q1^2),
 *             phi = q1 + (beta-1)(q1-1)^2                          eq. adim:q
 *   source    psi = dt~ (0, lap(q2/q1), lap(q3/q1))                eq. adim:q
 *   one step  fill ghosts; x1 sweep; fill ghosts; x2 sweep (entries 2 and 3
 *             swapped); fill ghosts; source by a second-order central
 *             difference, forward Euler                           eqs. fs:*
 *   sweep     Q_i -= dt/dx (A-dQ_{i+1/2} + A+dQ_{i-1/2})
 *                  - dt/dx (F~_{i+1/2} - F~_{i-1/2})               eq. fv-hr
 *   dt        dt_{n+1} = nu_W dx / max|s| of step n                 section 4
 *
 * Readings where the paper is silent:
 *   - the source uses lap(q2/q1), the Laplacian of the velocity z2;
 *   - the CFL maximum is over |s|, over the faces of the domain cells only;
 *   - two ghost layers, refilled from the current state before every
 *     sub-step; driven borders are evaluated at t_n for all three sub-steps;
 *   - Godunov splitting x1 -> x2 -> source in every step, one dt (or, on
 *     request, Strang's symmetric form x1(dt/2) -> x2 -> source -> x1(dt/2),
 *     a second-order variant of the consecutive application that section 3
 *     describes; the paper does not say which order it uses);
 *   - if W.W == 0 the limited wave is zero; at s == 0 the upwind side is i+1;
 *   - dt_0 comes from a speed-only pass over Q^0; a step that would pass
 *     t_end is shortened to end on it; nu_n > nu_max is an error, not a retry.
 *
 * The eigenvectors are not printed in the paper ("obtained in
 * straightforward fashion", section 3.2).  For the Roe matrix of section 3.2,
 * written with u = Z2/Z1, v = Z3/Z1 and c = sqrt(u^2 - 2 Z2 u + Phi):
 *   r1 = (1, s1, v (s1 - 2 Z2)/c),  r2 = (1, s2, v (2 Z2 - s2)/c),  r3 = (0,0,1)
 * The wave strengths solve dQ = a1 r1 + a2 r2 + a3 r3 (section 3.1).
 *
 * Arithmetic is IEEE binary64, compiled with -ffp-contract=off so that every
 * product and sum is rounded exactly as written.
 *
 * Axisymmetric mode (not in the paper, which is 2D Cartesian): x1 = z (axis),
 * x2 = r (radius, r_j = y0 + (j + 1/2) dx).  The source sub-step then adds the
 * cylindrical terms of div(rho u) and div(rho0 u u + p I):
 *   -(1/r) (q3, z2 z3, z3^2)    with z = q / q1,
 * and uses the cylindrical vector Laplacian of the velocity for the viscous
 * part (axial: d_zz + d_rr + (1/r) d_r; radial: d_zz + d_rr + (1/r) d_r - 1/r^2).
 * The two radial faces nearest the axis (r = 0 and r = dx) use the
 * first-order flux: with the second-order correction there, the spectral
 * radius of the linearised step exceeds one; with it removed the step is
 * stable up to CFL 0.5 (measured on the linearised oracle step).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG 2
#define AXIS_FACES 2  /* radial faces next to the axis with a first-order flux */

enum { BC_PERIODIC = 0, BC_EXTRAP = 1, BC_REFLECT = 2, BC_TAYLOR = 3, BC_HIFU = 4 };
enum { LIM_MC = 0, LIM_NONE = 1, LIM_LW = 2 };
enum { ST_NONREAL = 1, ST_CFL = 2, ST_NAN = 4 };

/* Parameters of one run.  Mirrored field by field by the Python wrapper. */
typedef struct {
  int nx, ny;
  int bc[4];          /* x-low, x-high, y-low, y-high */
  int limiter;        /* LIM_* */
  int sweeps;         /* bit 0: x1 sweep, bit 1: x2 sweep, bit 2: source */
  int geometry;       /* 0 Cartesian, 1 axisymmetric (x1 = z, x2 = r) */
  int envelope;       /* HIFU drive envelope: 0 one-sided turn-on, 1 packet */
  double beta;        /* 1 + B/2A */
  double delta;       /* dimensionless diffusivity dt~ = delta/(c0 L) */
  double dx;          /* cell size (dimensionless) */
  double nu_w;        /* wished CFL number */
  double nu_max;      /* largest accepted CFL number */
  double dt_fixed;    /* > 0: use this dt every step instead of the CFL rule */
  double x0, y0;      /* coordinates of the lower-left corner of cell (0,0) */
  double t0;          /* initial time */
  double taylor_ratio;/* dt~/beta of the Taylor-shock border (eq. OurTaylorS) */
  double taylor_angle;/* propagation angle theta_T of the Taylor shock */
  double amp;         /* HIFU drive amplitude A (eq. hifuBC) */
  double focal;       /* focal length F */
  double aperture;    /* half aperture a */
  int splitting;      /* 0: Godunov x1, x2, source; 1: Strang x1(dt/2), x2, source, x1(dt/2) */
  int reserved;
} ora_params;

typedef struct {
  ora_params p;
  int sx, sy;          /* padded extents nx + 2 NG, ny + 2 NG */
  double *q[3];
  double t;
  double dt;           /* dt given by the CFL rule (or dt_fixed) for the next step */
  double dt_last;      /* dt actually taken by the last step */
  long step;
  double smax;         /* max |s| of the last step */
  double nu_min, nu_max_seen, nu_mean, nu_m2;   /* Welford running mean / M2 */
  long nu_count;
  int status;
  int sweep_dir;       /* direction of the sweep in progress */
} ora_state;

/* max that propagates NaN, so that a NaN speed is never hidden */
static double max_nan(double a, double b) {
  if (a != a || b != b) return a != a ? a : b;
  return a > b ? a : b;
}

static size_t idx(const ora_state *st, int i, int j) {
  return (size_t)(j + NG) * (size_t)st->sx + (size_t)(i + NG);
}

/* ---------------------------------------------------------------------------
 * Driven borders.
 * Taylor shock (eq. OurTaylorS, rotated by theta_T as in section 4.1):
 *   q1 = 1 - (dt~/beta) tanh(x cos th + y sin th - t),
 *   (q2, q3) = (q1 - 1)(cos th, sin th).
 * HIFU drive (eq. hifuBC) on the x-low border for 0 <= x2 <= a:
 *   q1 = 1 + g, q2 = F g / sqrt(x2^2 + F^2), q3 = -x2 g / sqrt(x2^2 + F^2),
 *   g = A sin(2 pi tau) E(tau),  tau = t + x2^2/(2F) - x1,
 * with x1 the (negative) ghost-cell abscissa, i.e. linear propagation between
 * the border and the ghost centre.  E is read as a one-sided turn-on
 * exp(-(tau/4)^-10) for tau > 0 (0 otherwise) or as the packet
 * exp(-(tau/4)^10).
 * ------------------------------------------------------------------------- */
static void taylor_value(const ora_params *p, double x, double y, double t, double out[3]) {
  double ct = cos(p->taylor_angle), sn = sin(p->taylor_angle);
  double q1 = 1.0 - p->taylor_ratio * tanh(x * ct + y * sn - t);
  out[0] = q1;
  out[1] = (q1 - 1.0) * ct;
  out[2] = (q1 - 1.0) * sn;
}

static double hifu_envelope(int kind, double tau) {
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

static void hifu_value(const ora_params *p, double x1, double x2, double t, double out[3]) {
  const double two_pi = 6.283185307179586;
  double tau = t + x2 * x2 / (2.0 * p->focal) - x1;
  double g = p->amp * sin(two_pi * tau) * hifu_envelope(p->envelope, tau);
  double rn = sqrt(x2 * x2 + p->focal * p->focal);
  out[0] = 1.0 + g;
  out[1] = p->focal * g / rn;
  out[2] = -x2 * g / rn;
}

/* Fill every ghost cell from the current state.  Rows first (x ghosts of the
 * rows 0..ny-1), then columns (y ghosts of all columns, ghost columns
 * included).  Reflection mirrors cell -1-k onto k and negates the normal
 * momentum.  Corner ghosts are filled but no sub-step reads them. */
static void fill_ghosts(ora_state *st, double t) {
  const ora_params *p = &st->p;
  int nx = p->nx, ny = p->ny;
  for (int j = 0; j < ny; j++) {
    double yc = p->y0 + (j + 0.5) * p->dx;
    for (int g = 1; g <= NG; g++) {
      /* x-low ghost i = -g, x-high ghost i = nx - 1 + g */
      for (int side = 0; side < 2; side++) {
        int i = side == 0 ? -g : nx - 1 + g;
        int type = p->bc[side];
        double v[3];
        double xc = p->x0 + (i + 0.5) * p->dx;
        if (type == BC_PERIODIC) {
          int src = side == 0 ? i + nx : i - nx;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, src, j)];
        } else if (type == BC_REFLECT) {
          int src = side == 0 ? -1 - i : 2 * nx - 1 - i;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, src, j)];
          v[1] = -v[1];
        } else if (type == BC_TAYLOR) {
          taylor_value(p, xc, yc, t, v);
        } else if (type == BC_HIFU && side == 0 && yc >= 0.0 && yc <= p->aperture) {
          hifu_value(p, xc, yc, t, v);
        } else { /* extrapolation, and the HIFU border outside the aperture */
          int src = side == 0 ? 0 : nx - 1;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, src, j)];
        }
        for (int k = 0; k < 3; k++) st->q[k][idx(st, i, j)] = v[k];
      }
    }
  }
  for (int i = -NG; i < nx + NG; i++) {
    double xc = p->x0 + (i + 0.5) * p->dx;
    for (int g = 1; g <= NG; g++) {
      for (int side = 0; side < 2; side++) {
        int j = side == 0 ? -g : ny - 1 + g;
        int type = p->bc[2 + side];
        double v[3];
        double yc = p->y0 + (j + 0.5) * p->dx;
        if (type == BC_PERIODIC) {
          int src = side == 0 ? j + ny : j - ny;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, i, src)];
        } else if (type == BC_REFLECT) {
          int src = side == 0 ? -1 - j : 2 * ny - 1 - j;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, i, src)];
          v[2] = -v[2];
        } else if (type == BC_TAYLOR) {
          taylor_value(p, xc, yc, t, v);
        } else {
          int src = side == 0 ? 0 : ny - 1;
          for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, i, src)];
        }
        for (int k = 0; k < 3; k++) st->q[k][idx(st, i, j)] = v[k];
      }
    }
  }
}

/* ---------------------------------------------------------------------------
 * Roe solver for one interface of the x1 sweep (section 3.2).
 * qL, qR = (q1, q_normal, q_transverse).  Outputs the speeds s^p (eqs.
 * lambda1-lambda3) and the waves W^p = alpha^p r^p (section 3.1).
 * Returns 1 if the radicand of eqs. lambda1/lambda2 is negative.
 * ------------------------------------------------------------------------- */
int ora_roe(double beta, const double qL[3], const double qR[3], double s[3], double W[3][3]) {
  /* parameter vector z = (q1, q2/q1, q3/q1) of both cells */
  double rL = 1.0 / qL[0];
  double rR = 1.0 / qR[0];
  double zL2 = qL[1] * rL, zL3 = qL[2] * rL;
  double zR2 = qR[1] * rR, zR3 = qR[2] * rR;
  /* Roe average: arithmetic mean of Z_i and Z_{i-1} */
  double Z1 = 0.5 * (qL[0] + qR[0]);
  double Z2 = 0.5 * (zL2 + zR2);
  double Z3 = 0.5 * (zL3 + zR3);
  double Phi = 1.0 + 2.0 * (beta - 1.0) * (Z1 - 1.0);
  double rZ1 = 1.0 / Z1;
  double u = Z2 * rZ1;
  double v = Z3 * rZ1;
  /* radicand of eqs. lambda1, lambda2: (Z2/Z1)^2 - 2 (Z2)^2/Z1 + Phi */
  double D = u * u - 2.0 * Z2 * u + Phi;
  int nonreal = D < 0.0;
  double c = sqrt(D);
  s[0] = u + c;
  s[1] = u - c;
  s[2] = u;
  /* eigenvectors and wave strengths */
  double rc = 1.0 / c;
  double h = 0.5 * rc;
  double d1 = qR[0] - qL[0];
  double d2 = qR[1] - qL[1];
  double d3 = qR[2] - qL[2];
  double r13 = v * (s[0] - 2.0 * Z2) * rc;
  double r23 = v * (2.0 * Z2 - s[1]) * rc;
  double a1 = (d2 - s[1] * d1) * h;
  double a2 = (s[0] * d1 - d2) * h;
  double a3 = d3 - a1 * r13 - a2 * r23;
  W[0][0] = a1; W[0][1] = a1 * s[0]; W[0][2] = a1 * r13;
  W[1][0] = a2; W[1][1] = a2 * s[1]; W[1][2] = a2 * r23;
  W[2][0] = 0.0; W[2][1] = 0.0;      W[2][2] = a3;
  return nonreal;
}

/* The MC limiter (eq. limiter), its Godunov (phi = 0) and Lax-Wendroff
 * (phi = 1) special cases. */
static double limiter_phi(int kind, double theta) {
  if (kind == LIM_NONE) return 0.0;
  if (kind == LIM_LW) return 1.0;
  double a = 0.5 * (1.0 + theta);
  double m = a < 2.0 ? a : 2.0;
  double b = 2.0 * theta;
  m = m < b ? m : b;
  return m > 0.0 ? m : 0.0;
}

/* One 1D high-resolution update of a line of n cells with NG ghosts on each
 * side (eq. fv-hr).  line[k][c], c = 0..n+3, k = (q1, q_normal, q_transverse).
 * Returns max |s| over the n+1 faces of the domain cells. */
static double sweep_line(ora_state *st, int n, double *line[3], double lam) {
  int m_count = n + 2 * NG;           /* interfaces m = 1..n+3 between c-1, c */
  double (*s)[3] = calloc((size_t)m_count + 1, sizeof *s);
  double (*W)[3][3] = calloc((size_t)m_count + 1, sizeof *W);
  double (*amdq)[3] = calloc((size_t)m_count + 1, sizeof *amdq);
  double (*apdq)[3] = calloc((size_t)m_count + 1, sizeof *apdq);
  double (*F)[3] = calloc((size_t)m_count + 1, sizeof *F);
  double smax = 0.0;
  for (int m = 1; m < m_count; m++) {
    double qL[3], qR[3];
    for (int k = 0; k < 3; k++) { qL[k] = line[k][m - 1]; qR[k] = line[k][m]; }
    if (ora_roe(st->p.beta, qL, qR, s[m], W[m])) st->status |= ST_NONREAL;
  }
  for (int m = NG; m <= n + NG; m++) {
    /* fluctuations, eqs. fluc:m and fluc:p */
    for (int k = 0; k < 3; k++) {
      double am = 0.0, ap = 0.0;
      for (int p = 0; p < 3; p++) {
        double sm = s[m][p] < 0.0 ? s[m][p] : 0.0;
        double sp = s[m][p] > 0.0 ? s[m][p] : 0.0;
        am = am + sm * W[m][p][k];
        ap = ap + sp * W[m][p][k];
      }
      amdq[m][k] = am;
      apdq[m][k] = ap;
    }
    /* limited correction flux, eq. limiter */
    double coef[3];
    /* axisymmetric form: first-order (Godunov) flux on the radial faces at
     * r = 0 and r = dx, where the split geometric source otherwise makes the
     * second-order correction slightly unstable */
    int axis_face = st->p.geometry == 1 && st->sweep_dir == 1 && st->p.y0 == 0.0 &&
                    (m - NG) < AXIS_FACES;
    for (int p = 0; p < 3; p++) {
      int up = s[m][p] > 0.0 ? m - 1 : m + 1;
      double wdotw = W[m][p][0] * W[m][p][0] + W[m][p][1] * W[m][p][1] + W[m][p][2] * W[m][p][2];
      double wup = W[up][p][0] * W[m][p][0] + W[up][p][1] * W[m][p][1] + W[up][p][2] * W[m][p][2];
      double theta = wdotw > 0.0 ? wup / wdotw : 0.0;
      double phi = wdotw > 0.0 ? limiter_phi(st->p.limiter, theta) : 0.0;
      double as = fabs(s[m][p]);
      coef[p] = axis_face ? 0.0 : as * (1.0 - lam * as) * phi;
    }
    for (int k = 0; k < 3; k++)
      F[m][k] = 0.5 * (coef[0] * W[m][0][k] + coef[1] * W[m][1][k] + coef[2] * W[m][2][k]);
    for (int p = 0; p < 3; p++) smax = max_nan(smax, fabs(s[m][p]));
  }
  /* cell update: cell c has its left face at m = c and right face at c + 1 */
  for (int c = NG; c < n + NG; c++)
    for (int k = 0; k < 3; k++)
      line[k][c] = line[k][c] - lam * (amdq[c + 1][k] + apdq[c][k]) - lam * (F[c + 1][k] - F[c][k]);
  free(s); free(W); free(amdq); free(apdq); free(F);
  return smax;
}

/* x1 sweep (dir 0) or x2 sweep (dir 1, entries 2 and 3 swapped, section 3.2). */
static double sweep(ora_state *st, int dir, double lam) {
  int nx = st->p.nx, ny = st->p.ny;
  int n = dir == 0 ? nx : ny;
  int lines = dir == 0 ? ny : nx;
  int len = n + 2 * NG;
  int comp[3] = {0, dir == 0 ? 1 : 2, dir == 0 ? 2 : 1};
  double *buf = malloc(sizeof(double) * 3 * (size_t)len);
  double *line[3] = {buf, buf + len, buf + 2 * len};
  double smax = 0.0;
  st->sweep_dir = dir;
  for (int l = 0; l < lines; l++) {
    for (int c = 0; c < len; c++) {
      size_t id = dir == 0 ? idx(st, c - NG, l) : idx(st, l, c - NG);
      for (int k = 0; k < 3; k++) line[k][c] = st->q[comp[k]][id];
    }
    smax = max_nan(smax, sweep_line(st, n, line, lam));
    for (int c = NG; c < n + NG; c++) {
      size_t id = dir == 0 ? idx(st, c - NG, l) : idx(st, l, c - NG);
      for (int k = 0; k < 3; k++) st->q[comp[k]][id] = line[k][c];
    }
  }
  free(buf);
  return smax;
}

/* max |s| over all faces of the domain cells, both directions, no update. */
static double speed_pass(ora_state *st) {
  int nx = st->p.nx, ny = st->p.ny;
  double smax = 0.0;
  for (int dir = 0; dir < 2; dir++) {
    int n = dir == 0 ? nx : ny, lines = dir == 0 ? ny : nx;
    int comp[3] = {0, dir == 0 ? 1 : 2, dir == 0 ? 2 : 1};
    for (int l = 0; l < lines; l++)
      for (int c = 0; c <= n; c++) {
        double qL[3], qR[3], s[3], W[3][3];
        size_t iL = dir == 0 ? idx(st, c - 1, l) : idx(st, l, c - 1);
        size_t iR = dir == 0 ? idx(st, c, l) : idx(st, l, c);
        for (int k = 0; k < 3; k++) { qL[k] = st->q[comp[k]][iL]; qR[k] = st->q[comp[k]][iR]; }
        if (ora_roe(st->p.beta, qL, qR, s, W)) st->status |= ST_NONREAL;
        for (int p = 0; p < 3; p++) smax = max_nan(smax, fabs(s[p]));
      }
  }
  return smax;
}

/* Source sub-step (eq. fs:source): forward Euler with the 5-point Laplacian
 * of the velocity z = (q2/q1, q3/q1); axisymmetric terms in that mode. */
static void source(ora_state *st, double dt) {
  const ora_params *p = &st->p;
  int nx = p->nx, ny = p->ny;
  size_t tot = (size_t)st->sx * (size_t)st->sy;
  double *z2 = malloc(sizeof(double) * tot);
  double *z3 = malloc(sizeof(double) * tot);
  for (size_t c = 0; c < tot; c++) {
    double r = 1.0 / st->q[0][c];
    z2[c] = st->q[1][c] * r;
    z3[c] = st->q[2][c] * r;
  }
  double dx = p->dx;
  double coef = dt * p->delta / (dx * dx);
  for (int j = 0; j < ny; j++) {
    for (int i = 0; i < nx; i++) {
      size_t c = idx(st, i, j);
      size_t w = idx(st, i - 1, j), e = idx(st, i + 1, j);
      size_t s_ = idx(st, i, j - 1), n_ = idx(st, i, j + 1);
      if (p->geometry == 0) {
        double L2 = (z2[w] + z2[e]) + (z2[s_] + z2[n_]) - 4.0 * z2[c];
        double L3 = (z3[w] + z3[e]) + (z3[s_] + z3[n_]) - 4.0 * z3[c];
        st->q[1][c] = st->q[1][c] + coef * L2;
        st->q[2][c] = st->q[2][c] + coef * L3;
      } else {
        /* r_j at the cell centre; terms written in the order of the comment
         * at the top of this file. */
        double r = p->y0 + (j + 0.5) * dx;
        double L2 = (z2[w] + z2[e]) + (z2[s_] + z2[n_]) - 4.0 * z2[c]
                  + (z2[n_] - z2[s_]) * (dx / (2.0 * r));
        double L3 = (z3[w] + z3[e]) + (z3[s_] + z3[n_]) - 4.0 * z3[c]
                  + (z3[n_] - z3[s_]) * (dx / (2.0 * r)) - z3[c] * (dx * dx / (r * r));
        double g1 = st->q[2][c] / r;
        double g2 = z2[c] * z3[c] / r;
        double g3 = z3[c] * z3[c] / r;
        st->q[0][c] = st->q[0][c] - dt * g1;
        st->q[1][c] = st->q[1][c] + coef * L2 - dt * g2;
        st->q[2][c] = st->q[2][c] + coef * L3 - dt * g3;
      }
    }
  }
  free(z2); free(z3);
}

/* ---------------------------------------------------------------------------
 * Public entry points (called from Python through ctypes).
 * ------------------------------------------------------------------------- */
ora_state *ora_create(const ora_params *p, const double *q0) {
  ora_state *st = calloc(1, sizeof *st);
  st->p = *p;
  st->sx = p->nx + 2 * NG;
  st->sy = p->ny + 2 * NG;
  size_t tot = (size_t)st->sx * (size_t)st->sy;
  for (int k = 0; k < 3; k++) {
    st->q[k] = calloc(tot, sizeof(double));
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++)
        st->q[k][idx(st, i, j)] = q0[(size_t)k * p->nx * p->ny + (size_t)j * p->nx + i];
  }
  st->t = p->t0;
  st->nu_min = 1e300;
  if (p->dt_fixed > 0.0) {
    st->dt = p->dt_fixed;
  } else {
    fill_ghosts(st, st->t);
    double s0 = speed_pass(st);
    st->dt = p->nu_w * p->dx / s0;
  }
  return st;
}

void ora_destroy(ora_state *st) {
  if (!st) return;
  for (int k = 0; k < 3; k++) free(st->q[k]);
  free(st);
}

/* Advance by up to max_steps steps, stopping when t reaches t_end (t_end <= t
 * means no time limit) or the status becomes nonzero.  Returns steps taken. */
long ora_run(ora_state *st, double t_end, long max_steps) {
  const ora_params *p = &st->p;
  long done = 0;
  int timed = t_end > st->t;
  while (done < max_steps && st->status == 0) {
    if (timed && !(st->t < t_end)) break;
    double dt = st->dt;
    int last = 0;
    if (timed && st->t + dt >= t_end) { dt = t_end - st->t; last = 1; }
    double lam = dt / p->dx;
    double smax = 0.0;
    const int strang = p->splitting == 1;
    if (p->sweeps & 1) {
      fill_ghosts(st, st->t);
      smax = max_nan(smax, sweep(st, 0, strang ? lam * 0.5 : lam));
    }
    if (p->sweeps & 2) {
      fill_ghosts(st, st->t);
      smax = max_nan(smax, sweep(st, 1, lam));
    }
    if (p->sweeps & 4) {
      fill_ghosts(st, st->t);
      source(st, dt);
    }
    if (strang && (p->sweeps & 1)) {
      fill_ghosts(st, st->t);
      smax = max_nan(smax, sweep(st, 0, lam * 0.5));
    }
    if (smax != smax) st->status |= ST_NAN;
    st->smax = smax;
    if (p->sweeps & 3) {
      double nu = dt * smax / p->dx;
      if (nu > p->nu_max) st->status |= ST_CFL;
      if (!last) { /* the clamped final step is left out of the statistics */
        if (nu < st->nu_min) st->nu_min = nu;
        if (nu > st->nu_max_seen) st->nu_max_seen = nu;
        st->nu_count += 1;
        double d = nu - st->nu_mean;
        st->nu_mean += d / (double)st->nu_count;
        st->nu_m2 += d * (nu - st->nu_mean);
      }
    }
    if (p->dt_fixed <= 0.0 && smax > 0.0) st->dt = p->nu_w * p->dx / smax;
    st->dt_last = dt;
    st->t = last ? t_end : st->t + dt;
    st->step += 1;
    done += 1;
  }
  return done;
}

/* Moving domain (section 4: in the second stage of a run the domain moves
 * with the wave).  The window moves by (kx, ky) whole cells: afterwards cell
 * (i, j) holds what was cell (i + kx, j + ky), and the lower-left corner
 * moved by (kx dx, ky dx).  A cell with no old counterpart comes in through
 * a border and takes what that border's rule gives at the current time t:
 * the Taylor shock its analytic value (eq. OurTaylorS) at the new cell
 * centre; periodic the wrapped old cell; every other rule the nearest old
 * cell (zero-order extrapolation).  A cell coming in through a corner takes
 * the analytic value if either border is a Taylor border, else both rules in
 * turn.  Returns 0, or -1 when |kx| >= nx or |ky| >= ny. */
int ora_shift(ora_state *st, int kx, int ky) {
  ora_params *p = &st->p;
  int nx = p->nx, ny = p->ny;
  if (kx <= -nx || kx >= nx || ky <= -ny || ky >= ny) return -1;
  double x0n = p->x0 + kx * p->dx;
  double y0n = p->y0 + ky * p->dx;
  size_t n = (size_t)nx * (size_t)ny;
  double *nq = malloc(sizeof(double) * 3 * n);
  for (int j = 0; j < ny; j++) {
    for (int i = 0; i < nx; i++) {
      int si = i + kx, sj = j + ky;
      int out_x = si < 0 || si >= nx, out_y = sj < 0 || sj >= ny;
      int bx = p->bc[si < 0 ? 0 : 1], by = p->bc[sj < 0 ? 2 : 3];
      double v[3];
      if ((out_x && bx == BC_TAYLOR) || (out_y && by == BC_TAYLOR)) {
        taylor_value(p, x0n + (i + 0.5) * p->dx, y0n + (j + 0.5) * p->dx, st->t, v);
      } else {
        if (out_x) {
          if (bx == BC_PERIODIC) si = si < 0 ? si + nx : si - nx;
          else si = si < 0 ? 0 : nx - 1;
        }
        if (out_y) {
          if (by == BC_PERIODIC) sj = sj < 0 ? sj + ny : sj - ny;
          else sj = sj < 0 ? 0 : ny - 1;
        }
        for (int k = 0; k < 3; k++) v[k] = st->q[k][idx(st, si, sj)];
      }
      for (int k = 0; k < 3; k++) nq[(size_t)k * n + (size_t)j * nx + i] = v[k];
    }
  }
  for (int k = 0; k < 3; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) st->q[k][idx(st, i, j)] = nq[(size_t)k * n + (size_t)j * nx + i];
  free(nq);
  p->x0 = x0n;
  p->y0 = y0n;
  return 0;
}

/* Border rule of one side (0: x1-low, 1: x1-high, 2: x2-low, 3: x2-high)
 * from the next sub-step on: section 4.2's second stage makes the driven
 * x1-low border a zero-order extrapolation. */
void ora_set_bc(ora_state *st, int side, int bc) { st->p.bc[side] = bc; }

/* Lower-left corner of the window: out[0] = x0, out[1] = y0. */
void ora_corner(const ora_state *st, double *out) {
  out[0] = st->p.x0;
  out[1] = st->p.y0;
}

/* Copy the domain cells out: q[k*nx*ny + j*nx + i]. */
void ora_get(const ora_state *st, double *q) {
  int nx = st->p.nx, ny = st->p.ny;
  for (int k = 0; k < 3; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        q[(size_t)k * nx * ny + (size_t)j * nx + i] = st->q[k][idx(st, i, j)];
}

/* scalars: t, dt, smax, nu_min, nu_max, nu_mean, nu_std, step, status */
void ora_scalars(const ora_state *st, double *out) {
  double n = st->nu_count > 0 ? (double)st->nu_count : 1.0;
  double mean = st->nu_mean;
  double var = st->nu_m2 / n;
  out[0] = st->t;
  out[1] = st->dt;
  out[2] = st->smax;
  out[3] = st->nu_count > 0 ? st->nu_min : 0.0;
  out[4] = st->nu_max_seen;
  out[5] = mean;
  out[6] = var > 0.0 ? sqrt(var) : 0.0;
  out[7] = (double)st->step;
  out[8] = (double)st->status;
}

/* One interface of the x1 sweep, for unit checks: s[3], W[9] (row = family),
 * amdq[3], apdq[3].  Returns the non-real flag. */
int ora_interface(double beta, const double *qL, const double *qR, double *s, double *W,
                  double *amdq, double *apdq) {
  double Wm[3][3];
  int nr = ora_roe(beta, qL, qR, s, Wm);
  for (int p = 0; p < 3; p++)
    for (int k = 0; k < 3; k++) W[3 * p + k] = Wm[p][k];
  for (int k = 0; k < 3; k++) {
    double am = 0.0, ap = 0.0;
    for (int p = 0; p < 3; p++) {
      double sm = s[p] < 0.0 ? s[p] : 0.0;
      double sp = s[p] > 0.0 ? s[p] : 0.0;
      am = am + sm * Wm[p][k];
      ap = ap + sp * Wm[p][k];
    }
    amdq[k] = am;
    apdq[k] = ap;
  }
  return nr;
}

/* The driven border values of eq. hifuBC at (x1, x2, t) with the parameters
 * amplitude, focal length and envelope kind, whether or not (x1, x2) lies in
 * the aperture (for the pins): out = (q1, q2, q3). */
void ora_drive(const ora_params *p, double x1, double x2, double t, double *out) {
  hifu_value(p, x1, x2, t, out);
}

/* Evaluate the limiter function (for the pins). */
double ora_limiter(int kind, double theta) { return limiter_phi(kind, theta); }
