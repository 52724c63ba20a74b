/*
 * fvna.h -- C ABI of the GB300 finite-volume nonlinear acoustics library.
 *
 * The library advances the dimensionless balance laws of Velasco-Segura &
 * Rendon (arXiv 1311.3004), section 3, eq. OurSysAdim:
 *     q_t + f_1(q)_x1 + f_2(q)_x2 = psi(q),
 *     q = (rho/rho0)(1, u1/c0, u2/c0)                              (eq. adim:q)
 * with the fractional-step method of eqs. fs:cl1, fs:cl2, fs:source: an x1
 * sweep, an x2 sweep (entries 2 and 3 switched, end of section 3.2) and the
 * dissipative source, each sweep being the high-resolution update of eq.
 * fv-hr with Roe-linearised waves (section 3.2), fluctuations (eqs. fluc:m,
 * fluc:p) and the MC-limited correction flux (eq. limiter).  The time step
 * follows the CFL rule at the start of section 4.
 *
 * Every step runs in hand-written CUDA kernels for sm_103a; nothing here falls
 * back to the CPU.  All entry points return FVNA_OK (0) or a negative error
 * code; no C++ exception crosses this boundary.  A context is used by one host
 * thread at a time.
 *
 * Data layout across the boundary.  A state is three planes of nx*ny binary64
 * values in the paper's total variables (q1, q2, q3), plane k at offset
 * k*nx*ny, row-major with x1 fastest: element (k, j, i) at k*nx*ny + j*nx + i.
 * The library keeps its own device copy (SoA planes, rows padded to 32
 * elements); in FVNA_FP32_PERT precision that copy holds (q1 - 1, q2, q3) in
 * binary32, and conversions happen on the device.
 */
#ifndef FVNA_H
#define FVNA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FVNA_OK            0
#define FVNA_ERR_ARG      -1  /* invalid argument (sizes, enums, NULL, ...) */
#define FVNA_ERR_CUDA     -2  /* a CUDA runtime call failed */
#define FVNA_ERR_OOM      -3  /* device allocation failed */
#define FVNA_ERR_NONREAL  -4  /* a Roe radicand was negative (section 3.2, S bound) */
#define FVNA_ERR_CFL      -5  /* a step ran with nu > nu_max (section 4) */
#define FVNA_ERR_NAN      -6  /* a wave speed was NaN */
#define FVNA_ERR_SIZE     -7  /* domain larger than a fixed-size scratch area allows */
#define FVNA_ERR_TIMEOUT  -8  /* a kernel gave up waiting for one of its own asynchronous
                                 copies (bounded wait; the run stops, the context stays usable) */

/* ---- enumerations ------------------------------------------------------ */
enum fvna_precision {
  FVNA_FP64 = 0,       /* binary64 total variables; rounding-identical to the reference formulas */
  FVNA_FP32_PERT = 1   /* binary32 perturbations (q1-1, q2, q3), binary64 dt and budgets */
};
enum fvna_geometry {
  FVNA_CARTESIAN = 0,     /* the paper's 2D Cartesian system */
  FVNA_AXISYMMETRIC = 1   /* x1 = z, x2 = r, with the cylindrical source terms */
};
enum fvna_limiter {
  FVNA_LIM_MC = 0,     /* monotonized central, eq. limiter */
  FVNA_LIM_NONE = 1,   /* no correction: Godunov (section 3.1) */
  FVNA_LIM_LW = 2      /* phi = 1: Lax-Wendroff (section 3.1) */
};
enum fvna_bc {
  FVNA_BC_PERIODIC = 0,  /* wrap around (needs n >= 3 cells in that direction) */
  FVNA_BC_EXTRAP = 1,    /* zero-order extrapolation (section 4.2) */
  FVNA_BC_REFLECT = 2,   /* mirror, normal momentum negated (section 4.2); n >= 3 */
  FVNA_BC_TAYLOR = 3,    /* Taylor-shock values of eq. OurTaylorS (section 4.1) */
  FVNA_BC_HIFU = 4       /* focused drive of eq. hifuBC on the x1-low border */
};
enum fvna_splitting {
  FVNA_SPLIT_GODUNOV = 0,  /* x1 sweep, x2 sweep, source, each over dt (section 3, eqs. fs:*) */
  FVNA_SPLIT_STRANG = 1    /* x1 sweep over dt/2, x2 sweep, source, x1 sweep over dt/2: the
                              symmetric (second-order) order of the same fractional steps */
};
enum fvna_field {
  FVNA_FIELD_Q = 0,         /* 3*nx*ny binary64 total variables */
  FVNA_FIELD_PRESSURE = 1,  /* nx*ny binary64 p'/(rho0 c0^2) = q1 - 1 (linear EOS, section 2) */
  FVNA_FIELD_BUDGET = 2,    /* 3 binary64: sum over cells of (q1-1, q2, q3) after the last step */
  FVNA_FIELD_STATS = 3,     /* one fvna_stats */
  FVNA_FIELD_CORNER = 4,    /* 2 binary64: the window's lower-left corner (x0, y0), moved by
                               fvna_shift */
  FVNA_FIELD_AXIS = 5,      /* nx binary64: p'/(rho0 c0^2) = q1 - 1 along row 0 (the x1 axis
                               of a domain whose x2-low border is a symmetry axis, section 4.2) */
  FVNA_FIELD_OUTFLOW = 6    /* 3 binary64: the boundary-flux budget (fvna_set_budgets) of
                               (q1, q2, q3), summed over the steps since it was switched on */
};

/* ---- configuration ----------------------------------------------------- */
typedef struct fvna_config {
  int precision;        /* enum fvna_precision */
  int geometry;         /* enum fvna_geometry */
  int limiter;          /* enum fvna_limiter */
  int sweeps;           /* bit 0: x1 sweep, bit 1: x2 sweep, bit 2: source; 7 = full step */
  double beta;          /* nonlinearity 1 + B/2A (eq. OurSystem) */
  double delta;         /* dimensionless diffusivity dt~ = delta/(c0 L) (eq. phi-tdelta) */
  double dx;            /* cell size dx1 = dx2 (section 4) */
  double nu_w;          /* wished CFL number nu_W (section 4) */
  double nu_max;        /* a step with nu > nu_max ends the run with FVNA_ERR_CFL */
  double dt_fixed;      /* > 0: use this dt for every step instead of the CFL rule */
  int steps_per_graph;  /* steps captured per CUDA graph replay; 0 = default (32) */
  int tile_x;           /* x1-sweep tile width (16, 32 or 64 cells per warp row; binary32 also
                           60: the x1 sweep with the lanes along x1); 0 = default (picked
                           from the domain sizes) */
  int tile_y;           /* x2-sweep tile height (rows per warp); 0 = default (binary64 64,
                           binary32 10: 16 marched rows, two whole 8-row chunks) */
  int compensated;      /* FVNA_FP32_PERT: 0 = the increments of eq. fv-hr summed and added
                           to the state in one fused multiply-add (one rounding of the sum;
                           the default), 1 = the state and the two increments summed with
                           error-free two-sums (each increment's product rounded first) */
  int splitting;        /* enum fvna_splitting */
  int wait_limit;       /* FVNA_FP32_PERT: polls a sweep kernel makes while it waits for one of
                           its own asynchronous tile copies before it gives up (the run then
                           stops with FVNA_ERR_TIMEOUT and the context stays usable); 0 = the
                           default (2^22 polls, a few seconds at most); a negative value gives
                           up before the first poll, to exercise that error path */
} fvna_config;

/* One domain.  Coordinates are those of the lower-left corner of cell (0,0);
 * cell (i,j) has its centre at (x0 + (i+1/2) dx, y0 + (j+1/2) dx). */
typedef struct fvna_domain {
  int nx, ny;           /* cells; >= 1 each */
  int bc[4];            /* enum fvna_bc for x1-low, x1-high, x2-low, x2-high */
  int envelope;         /* HIFU envelope: 0 one-sided turn-on, 1 packet */
  int reserved;
  double x0, y0;        /* lower-left corner */
  double t0;            /* initial time */
  double dt0;           /* > 0: dt of the first step (resuming a run); 0: from a speed pass */
  double taylor_ratio;  /* dt~/beta of the Taylor-shock border */
  double taylor_angle;  /* propagation angle theta_T of that border */
  double amp;           /* HIFU drive amplitude A */
  double focal;         /* HIFU focal length F */
  double aperture;      /* HIFU half aperture a (drive where 0 <= x2 <= a) */
} fvna_domain;

typedef struct fvna_stats {
  long long steps;      /* steps taken since init */
  double t;             /* current time */
  double dt;            /* dt the CFL rule gives for the next step */
  double dt_last;       /* dt of the last step */
  double smax;          /* max |s| of the last step */
  double nu_min, nu_max, nu_mean, nu_std;  /* CFL numbers of the unclamped steps */
  int status;           /* 0 or the first error code seen (FVNA_ERR_NONREAL, _CFL, _NAN) */
  int reserved;
} fvna_stats;

typedef struct fvna_ctx fvna_ctx;

/* fvna_init -- create a context holding n_domains independent domains that
 * advance together (one launch per sub-step covers all of them).
 *   cfg          configuration shared by all domains (borrowed, copied)
 *   doms         n_domains domain descriptions (borrowed, copied)
 *   q0           n_domains pointers, each to 3*nx*ny binary64 total variables
 *                laid out as described above (borrowed, copied)
 *   q0_on_device nonzero if the q0 pointers are device pointers
 *   stream       cudaStream_t the library enqueues on (borrowed; NULL = legacy default)
 *   out          receives the new context, or NULL on failure
 * The first dt comes from a speed-only pass over q0 (section 4), unless
 * cfg->dt_fixed > 0 or the domain's dt0 > 0 (a resumed run: pass the state,
 * t and the dt reported by FVNA_FIELD_STATS to continue bit for bit).  Returns FVNA_ERR_ARG for bad sizes or enums, FVNA_ERR_OOM
 * when device memory runs out, FVNA_ERR_CUDA on any other CUDA failure. */
int fvna_init(const fvna_config *cfg, int n_domains, const fvna_domain *doms,
              const double *const *q0, int q0_on_device, void *stream, fvna_ctx **out);

/* fvna_step -- enqueue nsteps full steps (asynchronous on the context's
 * stream; no time limit).  Errors found on the device are reported by the
 * next fvna_sync / fvna_run / fvna_fields call. */
int fvna_step(fvna_ctx *ctx, long long nsteps);

/* fvna_run -- advance until t reaches t_end (the step that would pass t_end is
 * shortened to end on it) or max_steps steps were taken, whichever comes
 * first; t_end <= current t means no time limit.  Blocks until done.  Returns
 * FVNA_OK or the first device status (FVNA_ERR_NONREAL, _CFL, _NAN); on such
 * an error the state is the one the failing step produced.  stats may be NULL;
 * with several domains it receives domain 0's statistics. */
int fvna_run(fvna_ctx *ctx, double t_end, long long max_steps, fvna_stats *stats);

/* fvna_sync -- wait for the context's stream; return the device status. */
int fvna_sync(fvna_ctx *ctx);

/* fvna_fields -- copy one quantity of one domain into a caller buffer of
 * `bytes` bytes (host or device, per dst_on_device); see enum fvna_field for
 * sizes.  Synchronises the stream.  FVNA_ERR_ARG if bytes is too small. */
int fvna_fields(fvna_ctx *ctx, int domain, int what, void *dst, size_t bytes, int dst_on_device);

/* fvna_shift -- move the window of one domain by (kx, ky) whole cells: the
 * moving domain of section 4 (in the second stage of a run the domain moves
 * with the wave).  Afterwards cell (i, j) holds what was cell (i + kx, j + ky)
 * and the corner (x0, y0) has moved by (kx dx, ky dx).  A cell with no old
 * counterpart enters through a border and takes what that border's rule
 * gives at the domain's current time: FVNA_BC_TAYLOR the analytic value of
 * eq. OurTaylorS at the new cell centre, FVNA_BC_PERIODIC the wrapped old
 * cell, any other rule the nearest old cell (zero-order extrapolation).  A
 * cell entering through a corner takes the analytic value if either border
 * is a Taylor border, else both rules in turn.  Enqueued on the context's
 * stream after the work already enqueued (asynchronous; errors of the two
 * kernels surface at the next synchronising call).  Returns FVNA_ERR_ARG for
 * a NULL context, a bad domain index, |kx| >= nx, |ky| >= ny, or ky != 0 in
 * the axisymmetric geometry (where x2 is the radius). */
int fvna_shift(fvna_ctx *ctx, int domain, int kx, int ky);

/* fvna_set_bc -- change the border rule of one side of one domain between
 * steps (side 0..3: x1-low, x1-high, x2-low, x2-high).  Section 4.2's second
 * stage turns the driven x1-low border into a zero-order extrapolation once
 * the packet is in the domain.  The change is enqueued on the context's
 * stream after the work already enqueued.  Returns FVNA_ERR_ARG for a bad
 * domain, side or rule, for a periodic rule left without its partner on the
 * opposite side (or the reverse), for a periodic or reflective rule across
 * fewer than 3 cells, and for a driven rule (FVNA_BC_TAYLOR, FVNA_BC_HIFU)
 * the domain was not created with on that side (its border buffers are sized
 * at fvna_init). */
int fvna_set_bc(fvna_ctx *ctx, int domain, int side, int bc);

/* fvna_run_moving -- a two-stage run with a moving domain (section 4): the
 * window of every domain stays at rest until its time t passes t1, then
 * follows the wave at velocity (vx, vy) (x1 and x2 units per unit time; for
 * a plane wave the unit sound speed times its direction).  The run proceeds
 * in chunks of `every` steps, each taken as by fvna_run(ctx, t_end, every);
 * after each chunk a domain whose window lags the target displacement
 * (round(vx (t - t1) / dx), round(vy (t - t1) / dx)) cells, counted from
 * where the window was when the context was created, is moved by the
 * difference with fvna_shift (the count includes the caller's own
 * fvna_shift calls).  Stops at t_end (with several domains, once the first of
 * them reaches it), after max_steps steps, or at the first device error, like
 * fvna_run (same return codes; stats as there).
 * FVNA_ERR_ARG if every < 1, or for a shift fvna_shift would refuse. */
int fvna_run_moving(fvna_ctx *ctx, double t_end, long long max_steps, double t1, double vx,
                    double vy, int every, fvna_stats *stats);

/* fvna_step_timed -- take one step with its kernels launched one by one (not
 * from the step graph), CUDA events recorded between them on the context's
 * stream, and block until it is done.  ms receives the device time of each
 * launch in milliseconds: ms[0] x1 sweep (a plain copy if that sweep is off), ms[1] x2
 * sweep + source, ms[2] dt update (with FVNA_SPLIT_STRANG: also the second
 * x1 sweep and the copy that ends the step).  The step is identical to one of
 * fvna_step.  Returns FVNA_OK or the device status after the step. */
int fvna_step_timed(fvna_ctx *ctx, float ms[3]);

/* fvna_autotune -- pick the sweep tile shapes for a set of domains.  Builds a
 * throwaway context from the same arguments as fvna_init for each candidate
 * (binary64: tile_x in {16, 32, 64}, tile_y in {8, 16, 32, 64, 128}; binary32:
 * tile_x in {16, 32, 64, 60}, tile_y in {10, 18, 26, 34, 42}), runs one warm-up graph of
 * trial_steps steps and times a second one with CUDA events on `stream`,
 * destroys it, and returns in *best a copy of *cfg with the fastest tile_x and
 * tile_y (ms_per_step, if not NULL, receives its time per step).  The
 * caller's q0 is only read.  Errors as fvna_init; FVNA_ERR_ARG if
 * trial_steps < 1 or best is NULL. */
int fvna_autotune(const fvna_config *cfg, int n_domains, const fvna_domain *doms,
                  const double *const *q0, int q0_on_device, void *stream, int trial_steps,
                  fvna_config *best, float *ms_per_step);

/* fvna_set_budgets -- switch the per-step boundary-flux budget on (1) or off
 * (0) for every domain of the context.  On, each step runs one small binary64
 * kernel before each sweep that adds dt/dx times the net numerical flux out
 * through the two border faces of every line, Fh(n-1/2) - Fh(-1/2) with
 * Fh(-1/2) = f(Q_0) - A+dQ + F~ and Fh(n-1/2) = f(Q_{n-1}) + A-dQ + F~ (eqs.
 * fv-hr, fluc:m, fluc:p, limiter): the sum of eq. fv-hr over a line's cells
 * telescopes to that difference because the fluctuations of an inner face
 * add up to the flux difference (eq. RoeCond).  With periodic and
 * zero-order-extrapolation borders the source's Laplacian sums to zero, so
 * FVNA_FIELD_BUDGET(t) = FVNA_FIELD_BUDGET(t_on) - FVNA_FIELD_OUTFLOW(t) up to
 * rounding; a reflective border adds the viscous momentum flux into the
 * wall, and the axisymmetric form its geometric volume terms, which the
 * budget does not hold.  Switching on resets the sums to zero; either way
 * the step graph is captured again on the next step.  FVNA_ERR_ARG for a
 * NULL context or another value of on. */
int fvna_set_budgets(fvna_ctx *ctx, int on);

/* fvna_launch_count -- kernels this context has enqueued so far (each kernel
 * node of a graph replay counts once). */
long long fvna_launch_count(const fvna_ctx *ctx);

/* fvna_destroy -- free the context and its device memory (NULL is a no-op). */
void fvna_destroy(fvna_ctx *ctx);

/* fvna_strerror -- static text for a status code. */
const char *fvna_strerror(int code);

/* fvna_last_cuda_error -- the CUDA runtime's text for the last CUDA error
 * behind an FVNA_ERR_CUDA or FVNA_ERR_OOM return in this process (static
 * storage, never NULL; "no error" if none).  Not part of the paper's method. */
const char *fvna_last_cuda_error(void);

/* fvna_riemann -- run the device Roe solver of one x1-sweep interface on n
 * host pairs (section 3.2; fluctuations of eqs. fluc:m, fluc:p), for checks.
 *   qL, qR   n*3 binary64 total variables (q1, q2, q3) of cells i-1 and i
 *   s        n*3 speeds s^1..s^3 (eqs. lambda1-lambda3)
 *   W        n*9 waves, W[9*k + 3*p + c] = component c of W^p
 *   amdq     n*3 left-going fluctuation A-dQ
 *   apdq     n*3 right-going fluctuation A+dQ
 * precision selects the binary64 or binary32-perturbation solver.  All
 * buffers are host memory.  Returns FVNA_OK, or FVNA_ERR_NONREAL if some
 * radicand was negative (outputs are still written). */
int fvna_riemann(int precision, double beta, int n, const double *qL, const double *qR,
                 double *s, double *W, double *amdq, double *apdq);

/* fvna_step_noalloc -- one binary64 step that allocates no memory.  The paper
 * has no counterpart: this is for callers that cannot allocate device memory
 * at run time (an application that hands out all device memory up front, a
 * locked-down allocator, a real-time loop that cannot afford cudaMalloc and
 * its implicit synchronisation).
 *   cfg       precision must be FVNA_FP64; geometry, limiter, sweeps, beta,
 *             delta and dx are used, the CFL fields are not (dt is given)
 *   dom       one domain (nx*ny <= FVNA_NOALLOC_MAX_CELLS)
 *   q_in      device pointer, 3*nx*ny binary64 total variables in the layout
 *             described at the top of this file (caller-owned, read only)
 *   q_out     device pointer, same layout (caller-owned); may equal q_in
 *   t, dt     time of the state and the step to take (driven borders use t)
 *   smax_out  host pointer or NULL: receives max|s| of the step, from which
 *             the caller picks its next dt
 *   stream    cudaStream_t to run on (NULL = legacy default stream)
 * The intermediate planes and bookkeeping live in one file-scope device array
 * of about 13 MB, which every GPU that loads this library keeps until the
 * process exits.  The first call on a device looks that array up and sets the
 * kernels' attributes, so make it before any stream capture; every call
 * blocks until its step is done.  All calls share the array and each call
 * clears what must start at zero, but calls that overlap on the GPU (two host
 * threads, or several streams) race on it.  Results equal those of
 * fvna_step with cfg->dt_fixed = dt, bit for bit.  The library cannot check
 * the type or size of the caller's buffers: they must hold 3*nx*ny binary64
 * values each on the current device.  Returns FVNA_OK, FVNA_ERR_ARG (the
 * checks of fvna_init, a non-finite t or dt, or cfg->splitting other than
 * FVNA_SPLIT_GODUNOV), FVNA_ERR_SIZE for a larger domain, FVNA_ERR_NONREAL /
 * FVNA_ERR_NAN from the step, or FVNA_ERR_CUDA. */
#define FVNA_NOALLOC_MAX_CELLS 524288
int fvna_step_noalloc(const fvna_config *cfg, const fvna_domain *dom, const double *q_in,
                      double *q_out, double t, double dt, double *smax_out, void *stream);

/* ---- three dimensions ---------------------------------------------------
 * The paper implements two dimensions and states that the equations of its
 * section 2 (eq. OurSystem) carry over directly to three (section 3 opening
 * and the conclusions).  These entry points advance one 3D domain of the
 * same balance laws with a third velocity component:
 *     q = (rho/rho0)(1, u1/c0, u2/c0, u3/c0)          (eq. adim:q in 3D)
 * by the fractional steps x1 sweep, x2 sweep, x3 sweep, source (eqs.
 * fs:cl1-fs:source with a third directional step), each sweep eq. fv-hr with
 * the Roe solver of section 3.2 extended by the fourth component (a second
 * transverse family moving at u) and the MC-limited correction of eq.
 * limiter; the source uses the 7-point Laplacian; dt follows section 4's CFL
 * rule over all three directions.  States cross the boundary as four planes
 * of nx*ny*nz binary64 total variables (q1, q2, q3, q4), field f, cell
 * (i, j, k) at f*nx*ny*nz + (k*ny + j)*nx + i.  In FVNA_FP32_PERT precision
 * the device copy holds (q1 - 1, q2, q3, q4) in binary32. */
typedef struct fvna_domain3 {
  int nx, ny, nz;       /* cells; >= 1 each (>= 3 across a periodic or reflective pair) */
  int bc[6];            /* x1-low, x1-high, x2-low, x2-high, x3-low, x3-high: FVNA_BC_PERIODIC
                           (in pairs), FVNA_BC_EXTRAP or FVNA_BC_REFLECT */
  int substeps;         /* 0: the full step; otherwise the sub-steps to take, bit 0 x1 sweep,
                           bit 1 x2 sweep, bit 2 x3 sweep, bit 3 source */
  double t0;            /* initial time */
  double dt0;           /* > 0: dt of the first step; 0: from a speed pass over q0 */
} fvna_domain3;

typedef struct fvna3_ctx fvna3_ctx;

/* fvna3_init -- create a 3D context.
 *   cfg   precision (FVNA_FP64 or FVNA_FP32_PERT), limiter, beta, delta, dx,
 *         nu_w, nu_max, dt_fixed, steps_per_graph and compensated as in 2D;
 *         geometry must be FVNA_CARTESIAN and splitting FVNA_SPLIT_GODUNOV;
 *         sweeps is not read (dom->substeps selects sub-steps); tile_y is
 *         the height of the x2/x3 sweeps' tiles (0: 64)
 *   dom   the domain (borrowed, copied)
 *   q0    4*nx*ny*nz binary64 total variables in the layout above (borrowed,
 *         copied; device memory if q0_on_device)
 *   stream cudaStream_t to enqueue on (borrowed; NULL = legacy default)
 * The first dt comes from a speed-only pass over q0 unless dt_fixed or dt0
 * is set.  Returns FVNA_OK, FVNA_ERR_ARG for bad sizes, enums or border
 * rules, FVNA_ERR_OOM or FVNA_ERR_CUDA; *out is NULL on failure. */
int fvna3_init(const fvna_config *cfg, const fvna_domain3 *dom, const double *q0, int q0_on_device,
               void *stream, fvna3_ctx **out);
/* fvna3_run -- advance until t_end (the last step shortened to end on it;
 * t_end <= t: no time limit) or max_steps steps; blocks.  Returns FVNA_OK or
 * the first device status (FVNA_ERR_NONREAL, _CFL, _NAN); stats may be NULL. */
int fvna3_run(fvna3_ctx *ctx, double t_end, long long max_steps, fvna_stats *stats);
/* fvna3_step_timed -- one step launched kernel by kernel with CUDA events
 * between the launches on the context's stream; blocks.  ms receives the
 * device time in milliseconds of ms[0] the x1 sweep, ms[1] the x2 sweep,
 * ms[2] the x3 sweep, ms[3] the source, ms[4] the dt update. */
int fvna3_step_timed(fvna3_ctx *ctx, float ms[5]);
/* fvna3_fields -- copy FVNA_FIELD_Q (4*nx*ny*nz binary64), FVNA_FIELD_PRESSURE
 * (nx*ny*nz binary64 q1 - 1) or FVNA_FIELD_STATS (one fvna_stats) into a
 * caller buffer of `bytes` bytes (host or device per dst_on_device);
 * synchronises the stream.  FVNA_ERR_ARG if bytes is too small. */
int fvna3_fields(fvna3_ctx *ctx, int what, void *dst, size_t bytes, int dst_on_device);
/* fvna3_launch_count -- kernels this context has enqueued so far. */
long long fvna3_launch_count(const fvna3_ctx *ctx);
/* fvna3_destroy -- free the context and its device memory (NULL is a no-op). */
void fvna3_destroy(fvna3_ctx *ctx);

/* ---- learned sub-grid correction (not in the paper) ----------------------
 * A small convolutional network applied to coarse runs: three 3x3
 * convolutions with zero padding, 3 -> 32 -> 32 -> 3 channels, ReLU after
 * the first two:  y[o,i,j] = b[o] + sum_c sum_{u,v} w[o,c,u,v] x[c,i+u-1,j+v-1].
 * Weights and hidden activations are bfloat16, accumulation is FP32 (tensor
 * cores); training keeps FP32 master weights.  Parameters are one flat FP32
 * vector: w1 (32x3x3x3), b1 (32), w2 (32x32x3x3), b2 (32), w3 (3x32x3x3),
 * b3 (3), weights ordered [out][in][row][col].  Network tensors are FP32
 * channel planes (batch, 3, h, w), device memory; hidden activations are
 * kept by the network between a forward and the matching backward. */
#define FVNA_NET_PARAMS 11011
typedef struct fvna_net fvna_net;

/* fvna_net_create -- allocate a network on the current device from host
 * parameters (FVNA_NET_PARAMS floats, copied). */
int fvna_net_create(const float *params, fvna_net **out);
/* fvna_net_params -- copy the parameters out (dst, host) and/or replace them (src, host). */
int fvna_net_params(fvna_net *net, float *dst, const float *src);
/* fvna_net_forward -- y = net(in_scale * x) for a batch; x, y device FP32
 * planes (batch, 3, h, w).  h1_out / h2_out (device, or NULL) receive the two
 * hidden activations as bfloat16 bit patterns, pixel-major with 32 channels
 * (batch, h, w, 32).  Blocks. */
int fvna_net_forward(fvna_net *net, int batch, int h, int w, const float *x, float in_scale,
                     float *y, unsigned short *h1_out, unsigned short *h2_out, void *stream);
/* fvna_net_backward -- gradients of sum(gy * y) w.r.t. the parameters for the
 * last forward (same x, batch and size); gy device FP32 planes; grads (device,
 * FVNA_NET_PARAMS floats, or NULL). */
int fvna_net_backward(fvna_net *net, int batch, int h, int w, const float *x, float in_scale,
                      const float *gy, float *grads, void *stream);
/* fvna_net_train_step -- one Adam step (lr, beta 0.9/0.999) on the mean squared
 * error between net(in_scale * x) and target (device FP32 planes) over the
 * pixels at least `margin` from the image edges (crops of a larger field:
 * their edges see zero padding the full field does not).  edges (device,
 * batch x 4 ints: top, bottom, left, right, or NULL) gives per-image margins
 * instead, 0 on the sides where a crop meets the field's own edge.  loss
 * (host, or NULL) receives the loss before the step. */
int fvna_net_train_step(fvna_net *net, int batch, int h, int w, const float *x, float in_scale,
                        const float *target, int margin, const int *edges, float lr, double *loss,
                        void *stream);
/* fvna_net_destroy -- free the network (NULL is a no-op). */
void fvna_net_destroy(fvna_net *net);
/* fvna_set_correction -- after every `every`-th step (counted since init) of a
 * single-domain FVNA_FP32_PERT context, add out_scale * net(in_scale *
 * (q1-1, q2, q3)) to the state, except on the cells within edge_band cells of
 * a domain edge (a network trained on crops with a loss margin has not learnt
 * them); net = NULL detaches.  The network is borrowed and must outlive its
 * use.  FVNA_ERR_ARG with FVNA_SPLIT_STRANG (the correction follows the
 * Godunov step it was trained on). */
int fvna_set_correction(fvna_ctx *ctx, fvna_net *net, float in_scale, float out_scale,
                        int every, int edge_band);

#ifdef __cplusplus
}
#endif

#endif /* FVNA_H */
