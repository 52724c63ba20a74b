/*
 * fvna_oracle3d.c -- plain, slow FP64 CPU oracle of the three-dimensional
 * form of the finite-volume scheme of Velasco-Segura & Rendon (arXiv
 * 1311.3004).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library, and the library never calls it.
 *
 * The paper implements two dimensions and states that its equations (section
 * 2, eq. OurSystem) carry over directly to three (section 3 opening, and the
 * conclusions).  Written for three dimensions in the variables of eq.
 * adim:q:
 *
 *   state     q = (q1, q2, q3, q4) = (rho/rho0)(1, u1/c0, u2/c0, u3/c0)
 *   flux      f_j = q^{j+1}/(q1)^2 ((q1)^2, q2, q3, q4) + phi (0, d1j, d2j, d3j),
 *             phi = q1 + (beta-1)(q1-1)^2
 *   source    psi = dt~ (0, lap(q2/q1), lap(q3/q1), lap(q4/q1))
 *   one step  fill ghosts; x1 sweep; fill ghosts; x2 sweep; fill ghosts; x3
 *             sweep; fill ghosts; source (7-point Laplacian, forward Euler):
 *             the fractional steps of eqs. fs:cl1-fs:source with a third
 *             directional step.  Each sweep is eq. fv-hr with the entries of
 *             the state permuted so that the normal momentum comes second:
 *             x1 (q1, q2, q3, q4), x2 (q1, q3, q2, q4), x3 (q1, q4, q2, q3).
 *
 * Roe solver of one x1 interface (section 3.2 with the parameter vector
 * z = (q1, q2/q1, q3/q1, q4/q1) and Z the arithmetic mean of the two cells'
 * z): the matrix of section 3.2 gains a fourth row
 *   (-2 Z2 Z4/Z1, Z4/Z1, 0, Z2/Z1),
 * so the eigenvalues are those of eqs. lambda1-lambda3 with lambda3 double
 * (two transverse families moving at u = Z2/Z1).  With v = Z3/Z1, w = Z4/Z1,
 * c = sqrt(u^2 - 2 Z2 u + Phi):
 *   r1 = (1, s1, v (s1 - 2 Z2)/c, w (s1 - 2 Z2)/c),
 *   r2 = (1, s2, v (2 Z2 - s2)/c, w (2 Z2 - s2)/c),
 *   r3 = (0, 0, 1, 0),  r4 = (0, 0, 0, 1)
 * (the fourth components solve row four of A r = s r exactly as the third
 * solves row three).  Wave strengths solve dQ = sum_p a_p r_p.  Fluctuations
 * (eqs. fluc:m, fluc:p), the MC-limited correction (eq. limiter, theta from
 * full four-component dot products) and the update are those of the 2D
 * oracle with a fourth component.
 *
 * Readings as in the 2D oracle (fvna_oracle.c): two ghost layers refilled
 * before every sub-step; zero-order extrapolation copies the edge cell; a
 * reflective border mirrors cell -1-k onto k and negates the normal momentum;
 * periodic borders wrap; max|s| over the faces of the domain cells in all
 * three directions gives dt_{n+1} = nu_W dx / max|s| (section 4).  The
 * Laplacian is summed as ((W + E) + (S + N) - 4 C) + ((B + T) - 2 C), so that
 * on a state that does not vary along x3 it is the 2D oracle's sum exactly.
 *
 * IEEE binary64, compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG3 2

enum { B3_PERIODIC = 0, B3_EXTRAP = 1, B3_REFLECT = 2 };
enum { L3_MC = 0, L3_NONE = 1, L3_LW = 2 };
enum { S3_NONREAL = 1, S3_CFL = 2, S3_NAN = 4 };

/* Parameters of one 3D run.  Mirrored field by field by the Python wrapper. */
typedef struct {
  int nx, ny, nz;
  int bc[6];          /* x1-low, x1-high, x2-low, x2-high, x3-low, x3-high */
  int limiter;        /* L3_* */
  int sweeps;         /* bit 0: x1, bit 1: x2, bit 2: x3, bit 3: source */
  double beta, delta, dx, nu_w, nu_max, dt_fixed, t0;
} ora3_params;

typedef struct {
  ora3_params p;
  int sx, sy, sz;      /* padded extents */
  double *q[4];
  double t, dt, dt_last, smax;
  long step;
  int status;
} ora3_state;

static double max_nan3(double a, double b) {
  if (a != a || b != b) return a != a ? a : b;
  return a > b ? a : b;
}

static size_t id3(const ora3_state *st, int i, int j, int k) {
  return ((size_t)(k + NG3) * (size_t)st->sy + (size_t)(j + NG3)) * (size_t)st->sx +
         (size_t)(i + NG3);
}

/* index of cell (a, b, c) where a runs along direction dir and (b, c) are the
 * other two coordinates in increasing axis order */
static size_t idd(const ora3_state *st, int dir, int a, int b, int c) {
  if (dir == 0) return id3(st, a, b, c);
  if (dir == 1) return id3(st, b, a, c);
  return id3(st, b, c, a);
}

static int extent(const ora3_params *p, int dir) {
  return dir == 0 ? p->nx : dir == 1 ? p->ny : p->nz;
}

/* Ghosts of direction dir for every line of the domain cells. */
static void fill_dir(ora3_state *st, int dir) {
  const ora3_params *p = &st->p;
  int n = extent(p, dir);
  int o1 = dir == 0 ? 1 : 0, o2 = dir == 2 ? 1 : 2;
  int n1 = extent(p, o1), n2 = extent(p, o2);
  for (int c = 0; c < n2; c++)
    for (int b = 0; b < n1; b++)
      for (int g = 1; g <= NG3; g++)
        for (int side = 0; side < 2; side++) {
          int a = side == 0 ? -g : n - 1 + g;
          int type = p->bc[2 * dir + side];
          int src;
          if (type == B3_PERIODIC) src = side == 0 ? a + n : a - n;
          else if (type == B3_REFLECT) src = side == 0 ? -1 - a : 2 * n - 1 - a;
          else src = side == 0 ? 0 : n - 1;
          for (int f = 0; f < 4; f++) {
            double v = st->q[f][idd(st, dir, src, b, c)];
            if (type == B3_REFLECT && f == 1 + dir) v = -v;
            st->q[f][idd(st, dir, a, b, c)] = v;
          }
        }
}

static void fill_ghosts3(ora3_state *st) {
  for (int d = 0; d < 3; d++) fill_dir(st, d);
}

/* Roe solver of one interface, state (q1, q_normal, q_t1, q_t2).  Returns 1
 * if the radicand is negative. */
int ora3_roe(double beta, const double qL[4], const double qR[4], double s[4], double W[4][4]) {
  double rL = 1.0 / qL[0];
  double rR = 1.0 / qR[0];
  double zL2 = qL[1] * rL, zL3 = qL[2] * rL, zL4 = qL[3] * rL;
  double zR2 = qR[1] * rR, zR3 = qR[2] * rR, zR4 = qR[3] * rR;
  double Z1 = 0.5 * (qL[0] + qR[0]);
  double Z2 = 0.5 * (zL2 + zR2);
  double Z3 = 0.5 * (zL3 + zR3);
  double Z4 = 0.5 * (zL4 + zR4);
  double Phi = 1.0 + 2.0 * (beta - 1.0) * (Z1 - 1.0);
  double rZ1 = 1.0 / Z1;
  double u = Z2 * rZ1;
  double v = Z3 * rZ1;
  double w = Z4 * rZ1;
  double D = u * u - 2.0 * Z2 * u + Phi;
  int nonreal = D < 0.0;
  double c = sqrt(D);
  s[0] = u + c;
  s[1] = u - c;
  s[2] = u;
  s[3] = u;
  double rc = 1.0 / c;
  double h = 0.5 * rc;
  double d1 = qR[0] - qL[0];
  double d2 = qR[1] - qL[1];
  double d3 = qR[2] - qL[2];
  double d4 = qR[3] - qL[3];
  double r13 = v * (s[0] - 2.0 * Z2) * rc;
  double r23 = v * (2.0 * Z2 - s[1]) * rc;
  double r14 = w * (s[0] - 2.0 * Z2) * rc;
  double r24 = w * (2.0 * Z2 - s[1]) * rc;
  double a1 = (d2 - s[1] * d1) * h;
  double a2 = (s[0] * d1 - d2) * h;
  double a3 = d3 - a1 * r13 - a2 * r23;
  double a4 = d4 - a1 * r14 - a2 * r24;
  W[0][0] = a1; W[0][1] = a1 * s[0]; W[0][2] = a1 * r13; W[0][3] = a1 * r14;
  W[1][0] = a2; W[1][1] = a2 * s[1]; W[1][2] = a2 * r23; W[1][3] = a2 * r24;
  W[2][0] = 0.0; W[2][1] = 0.0;      W[2][2] = a3;       W[2][3] = 0.0;
  W[3][0] = 0.0; W[3][1] = 0.0;      W[3][2] = 0.0;      W[3][3] = a4;
  return nonreal;
}

static double limiter3(int kind, double theta) {
  if (kind == L3_NONE) return 0.0;
  if (kind == L3_LW) return 1.0;
  double a = 0.5 * (1.0 + theta);
  double m = a < 2.0 ? a : 2.0;
  double b = 2.0 * theta;
  m = m < b ? m : b;
  return m > 0.0 ? m : 0.0;
}

/* eq. fv-hr on one line of n cells with NG3 ghosts per side; line[k][c],
 * c = 0..n+3.  Returns max |s| over the n+1 faces of the domain cells. */
static double sweep_line3(ora3_state *st, int n, double *line[4], double lam) {
  int m_count = n + 2 * NG3;
  double (*s)[4] = calloc((size_t)m_count + 1, sizeof *s);
  double (*W)[4][4] = calloc((size_t)m_count + 1, sizeof *W);
  double (*amdq)[4] = calloc((size_t)m_count + 1, sizeof *amdq);
  double (*apdq)[4] = calloc((size_t)m_count + 1, sizeof *apdq);
  double (*F)[4] = calloc((size_t)m_count + 1, sizeof *F);
  double smax = 0.0;
  for (int m = 1; m < m_count; m++) {
    double qL[4], qR[4];
    for (int k = 0; k < 4; k++) { qL[k] = line[k][m - 1]; qR[k] = line[k][m]; }
    if (ora3_roe(st->p.beta, qL, qR, s[m], W[m])) st->status |= S3_NONREAL;
  }
  for (int m = NG3; m <= n + NG3; m++) {
    for (int k = 0; k < 4; k++) {
      double am = 0.0, ap = 0.0;
      for (int p = 0; p < 4; p++) {
        double sm = s[m][p] < 0.0 ? s[m][p] : 0.0;
        double sp = s[m][p] > 0.0 ? s[m][p] : 0.0;
        am = am + sm * W[m][p][k];
        ap = ap + sp * W[m][p][k];
      }
      amdq[m][k] = am;
      apdq[m][k] = ap;
    }
    double coef[4];
    for (int p = 0; p < 4; p++) {
      int up = s[m][p] > 0.0 ? m - 1 : m + 1;
      double wdotw = 0.0, wup = 0.0;
      for (int k = 0; k < 4; k++) {
        wdotw = wdotw + W[m][p][k] * W[m][p][k];
        wup = wup + W[up][p][k] * W[m][p][k];
      }
      double theta = wdotw > 0.0 ? wup / wdotw : 0.0;
      double phi = wdotw > 0.0 ? limiter3(st->p.limiter, theta) : 0.0;
      double as = fabs(s[m][p]);
      coef[p] = as * (1.0 - lam * as) * phi;
    }
    for (int k = 0; k < 4; k++)
      F[m][k] = 0.5 * (coef[0] * W[m][0][k] + coef[1] * W[m][1][k] + coef[2] * W[m][2][k] +
                       coef[3] * W[m][3][k]);
    for (int p = 0; p < 4; p++) smax = max_nan3(smax, fabs(s[m][p]));
  }
  for (int c = NG3; c < n + NG3; c++)
    for (int k = 0; k < 4; k++)
      line[k][c] = line[k][c] - lam * (amdq[c + 1][k] + apdq[c][k]) - lam * (F[c + 1][k] - F[c][k]);
  free(s); free(W); free(amdq); free(apdq); free(F);
  return smax;
}

/* One directional sweep (dir 0, 1, 2), entries permuted so that the normal
 * momentum comes second. */
static double sweep3(ora3_state *st, int dir, double lam) {
  const ora3_params *p = &st->p;
  static const int comp[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
  int n = extent(p, dir);
  int o1 = dir == 0 ? 1 : 0, o2 = dir == 2 ? 1 : 2;
  int n1 = extent(p, o1), n2 = extent(p, o2);
  int len = n + 2 * NG3;
  double *buf = malloc(sizeof(double) * 4 * (size_t)len);
  double *line[4] = {buf, buf + len, buf + 2 * len, buf + 3 * len};
  double smax = 0.0;
  for (int c = 0; c < n2; c++)
    for (int b = 0; b < n1; b++) {
      for (int a = 0; a < len; a++) {
        size_t id = idd(st, dir, a - NG3, b, c);
        for (int k = 0; k < 4; k++) line[k][a] = st->q[comp[dir][k]][id];
      }
      smax = max_nan3(smax, sweep_line3(st, n, line, lam));
      for (int a = NG3; a < n + NG3; a++) {
        size_t id = idd(st, dir, a - NG3, b, c);
        for (int k = 0; k < 4; k++) st->q[comp[dir][k]][id] = line[k][a];
      }
    }
  free(buf);
  return smax;
}

/* max |s| over all faces of the domain cells, all directions, no update */
static double speed_pass3(ora3_state *st) {
  const ora3_params *p = &st->p;
  static const int comp[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
  double smax = 0.0;
  for (int dir = 0; dir < 3; dir++) {
    int n = extent(p, dir);
    int o1 = dir == 0 ? 1 : 0, o2 = dir == 2 ? 1 : 2;
    int n1 = extent(p, o1), n2 = extent(p, o2);
    for (int c = 0; c < n2; c++)
      for (int b = 0; b < n1; b++)
        for (int a = 0; a <= n; a++) {
          double qL[4], qR[4], s[4], W[4][4];
          size_t iL = idd(st, dir, a - 1, b, c), iR = idd(st, dir, a, b, c);
          for (int k = 0; k < 4; k++) {
            qL[k] = st->q[comp[dir][k]][iL];
            qR[k] = st->q[comp[dir][k]][iR];
          }
          if (ora3_roe(p->beta, qL, qR, s, W)) st->status |= S3_NONREAL;
          for (int q = 0; q < 4; q++) smax = max_nan3(smax, fabs(s[q]));
        }
  }
  return smax;
}

/* Source sub-step: forward Euler with the 7-point Laplacian of the velocity. */
static void source3(ora3_state *st, double dt) {
  const ora3_params *p = &st->p;
  size_t tot = (size_t)st->sx * st->sy * st->sz;
  double *z[3];
  for (int f = 0; f < 3; f++) z[f] = malloc(sizeof(double) * tot);
  for (size_t c = 0; c < tot; c++) {
    double r = 1.0 / st->q[0][c];
    for (int f = 0; f < 3; f++) z[f][c] = st->q[f + 1][c] * r;
  }
  double coef = dt * p->delta / (p->dx * p->dx);
  for (int k = 0; k < p->nz; k++)
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++) {
        size_t c = id3(st, i, j, k);
        size_t w = id3(st, i - 1, j, k), e = id3(st, i + 1, j, k);
        size_t s_ = id3(st, i, j - 1, k), n_ = id3(st, i, j + 1, k);
        size_t b = id3(st, i, j, k - 1), t = id3(st, i, j, k + 1);
        for (int f = 0; f < 3; f++) {
          double L = ((z[f][w] + z[f][e]) + (z[f][s_] + z[f][n_]) - 4.0 * z[f][c]) +
                     ((z[f][b] + z[f][t]) - 2.0 * z[f][c]);
          st->q[f + 1][c] = st->q[f + 1][c] + coef * L;
        }
      }
  for (int f = 0; f < 3; f++) free(z[f]);
}

ora3_state *ora3_create(const ora3_params *p, const double *q0) {
  ora3_state *st = calloc(1, sizeof *st);
  st->p = *p;
  st->sx = p->nx + 2 * NG3;
  st->sy = p->ny + 2 * NG3;
  st->sz = p->nz + 2 * NG3;
  size_t tot = (size_t)st->sx * st->sy * st->sz;
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (int f = 0; f < 4; f++) {
    st->q[f] = calloc(tot, sizeof(double));
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++)
          st->q[f][id3(st, i, j, k)] =
              q0[(size_t)f * n + ((size_t)k * p->ny + j) * p->nx + i];
  }
  st->t = p->t0;
  if (p->dt_fixed > 0.0) {
    st->dt = p->dt_fixed;
  } else {
    fill_ghosts3(st);
    st->dt = p->nu_w * p->dx / speed_pass3(st);
  }
  return st;
}

void ora3_destroy(ora3_state *st) {
  if (!st) return;
  for (int f = 0; f < 4; f++) free(st->q[f]);
  free(st);
}

/* Advance by up to max_steps steps, stopping at t_end (t_end <= t: no time
 * limit) or on a nonzero status.  Returns the steps taken. */
long ora3_run(ora3_state *st, double t_end, long max_steps) {
  const ora3_params *p = &st->p;
  long done = 0;
  int timed = t_end > st->t;
  while (done < max_steps && st->status == 0) {
    if (timed && !(st->t < t_end)) break;
    double dt = st->dt;
    int last = 0;
    if (timed && st->t + dt >= t_end) { dt = t_end - st->t; last = 1; }
    double lam = dt / p->dx;
    double smax = 0.0;
    for (int d = 0; d < 3; d++)
      if (p->sweeps & (1 << d)) {
        fill_ghosts3(st);
        smax = max_nan3(smax, sweep3(st, d, lam));
      }
    if (p->sweeps & 8) {
      fill_ghosts3(st);
      source3(st, dt);
    }
    if (smax != smax) st->status |= S3_NAN;
    st->smax = smax;
    if (p->sweeps & 7) {
      double nu = dt * smax / p->dx;
      if (nu > p->nu_max) st->status |= S3_CFL;
    }
    if (p->dt_fixed <= 0.0 && smax > 0.0) st->dt = p->nu_w * p->dx / smax;
    st->dt_last = dt;
    st->t = last ? t_end : st->t + dt;
    st->step += 1;
    done += 1;
  }
  return done;
}

void ora3_get(const ora3_state *st, double *q) {
  const ora3_params *p = &st->p;
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (int f = 0; f < 4; f++)
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++)
          q[(size_t)f * n + ((size_t)k * p->ny + j) * p->nx + i] = st->q[f][id3(st, i, j, k)];
}

/* scalars: t, dt, smax, step, status, dt_last */
void ora3_scalars(const ora3_state *st, double *out) {
  out[0] = st->t;
  out[1] = st->dt;
  out[2] = st->smax;
  out[3] = (double)st->step;
  out[4] = (double)st->status;
  out[5] = st->dt_last;
}

/* One x1 interface of the 3D solver, for unit checks: s[4], W[16] (row =
 * family), amdq[4], apdq[4].  Returns the non-real flag. */
int ora3_interface(double beta, const double *qL, const double *qR, double *s, double *W,
                   double *amdq, double *apdq) {
  double Wm[4][4];
  int nr = ora3_roe(beta, qL, qR, s, Wm);
  for (int p = 0; p < 4; p++)
    for (int k = 0; k < 4; k++) W[4 * p + k] = Wm[p][k];
  for (int k = 0; k < 4; k++) {
    double am = 0.0, ap = 0.0;
    for (int p = 0; p < 4; p++) {
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
