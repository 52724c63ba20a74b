// fvna_types.h -- structures shared by the host runtime and the kernels.
#pragma once

#include <stdint.h>

namespace fvna {

enum { BC_PERIODIC = 0, BC_EXTRAP = 1, BC_REFLECT = 2, BC_TAYLOR = 3, BC_HIFU = 4 };
enum { LIM_MC = 0, LIM_NONE = 1, LIM_LW = 2 };
// ST_TIMEOUT: a kernel gave up waiting for one of its own asynchronous copies
enum { ST_NONREAL = 1, ST_CFL = 2, ST_NAN = 4, ST_TIMEOUT = 8 };

// Halo widths: the x1 sweep reads 2 cells beyond its tile (the limiter looks
// one interface upwind), the x2 sweep with the fused source reads 3.
constexpr int HALO_X = 2;
constexpr int HALO_Y = 3;
// Axisymmetric form: radial faces next to the axis that use the first-order
// flux (r = 0 and r = dx).
constexpr int AXIS_FACES = 2;
// Columns a warp of the x2 sweep updates (lanes 1..30; lanes 0 and 31 carry
// the neighbour columns the source's Laplacian needs).
constexpr int YCOLS = 30;
// Rows of one x1-sweep warp tile (one lane per row).
constexpr int XROWS = 32;

// One domain as the kernels see it (read-only during a step).
struct DomDev {
  int nx, ny, pitch, env;       // sizes, row pitch in elements, HIFU envelope kind
  int bc[4];                    // x-low, x-high, y-low, y-high
  double x0, y0;                // lower-left corner
  double taylor_ratio, taylor_ct, taylor_st;
  double amp, focal, aperture;
  double dt0;                   // > 0: first dt given by the caller
  void *qa[3];                  // state planes (start and end of every step)
  void *qb[3];                  // planes after the x1 sweep
  void *drive;                  // HIFU border values of the current step, 3 planes of
                                // HALO_Y x ny (ghost column -1-k at k*ny + row), or NULL
  void *ghost32;                // binary32 domains with a driven border: the ghost ring
                                // (fvna_sweeps32.cuh), or NULL
};

// Per-domain scalars that evolve on the device (one step = K1, K2, K3).
struct DomScal {
  double t, dt, dt_cfl, dt_last, t_end;
  double smax_last;
  double nu_min, nu_max, nu_mean, nu_m2;
  long long nu_count;
  long long step, steps_left;
  unsigned long long smax_bits;  // atomic max of |s| during the current step
  int status_bits;               // ST_* raised by the sweeps of the current step
  int status;                    // sticky ST_* of the run
  int done, last, timed, pad;
  double budget_acc[3];          // sum over cells of the state after the step (accumulating)
  double budget[3];              // the same, for the last completed step
  // per-step constants derived from dt (set wherever dt is set)
  double lam, coef;              // dt/dx and dt*delta/dx^2
  float lam32, coef32, dt32, pad32;
  // binary64 boundary-flux budget (fvna_set_budgets): sum over the sweeps of
  // dt/dx times the net numerical flux out through the domain's border faces
  double outflow[3];
};

// One warp's work item: domain, the tile origin (cells) and, for the
// binary32 x2 sweep, the tile's height (0: the sweep's tile_y).
struct Tile {
  int dom, x0, y0, pad;
};

// Arguments of every step kernel.
struct StepArgs {
  const DomDev *doms;
  DomScal *scal;
  const Tile *tiles;
  int ntiles;
  int ndom;
  double beta, delta, dx, nu_w, nu_max, dt_fixed;
  int limiter, geometry, sweeps, tile_y;
  int compensated;               // binary32 update with error-free two-sums
  int x_half;                    // 1: the x1 sweep advances dt/2 (Strang splitting)
  const void *tmaps;             // binary32 sweeps: TMA tensor maps, one set per domain
  unsigned *counters;            // binary32 sweeps: next-tile counters of the x1 and x2 sweeps
  int sweep;                     // 0: x1 sweep, 1: x2 sweep
  int *redo;                     // binary32 x2 sweep: redo[1] counts the tiles listed for
                                 // the general split, listed from redo[redo_off] on
  int redo_off;
  int fold_advance;              // binary32 x2 sweep: its last block ends the step
                                 // (k_advance's work; arrivals counted in counters[2])
  int wait_polls;                // binary32 sweeps: polls of a first wait for a tile copy
                                 // before giving up (0: give up at once)
};

}  // namespace fvna
