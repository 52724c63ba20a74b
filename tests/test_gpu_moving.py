"""Moving domain on the GPU (section 4: in the second stage of a run the
domain moves with the wave), through the C ABI, against the CPU oracle, and
the Taylor-shock study of section 4.1 (Table tab:error-ts) run on it.

- fvna_shift between steps matches the oracle's shift bit for bit in
  binary64 (periodic, extrapolation and reflective borders), and the
  binary32 form within its bar;
- fvna_run_moving follows a rotated Taylor shock like the oracle's moving
  run (driven borders: a few ulp of the total state);
- a moving window that follows the shock to t = 100 reproduces the paper's
  error table at theta_T = 0: E_1 falls with eta at an order above one and
  lies at eta = 82 within a factor of three of the printed best..worst range.
  At the rotated angles the analytic Dirichlet borders (the paper's) cut the
  shock front and set the error, which shrinks as the window widens across
  the propagation direction; on windows 100 units wide (the paper ran its
  moving domains 100 wavelengths long) the rotated errors converge at the
  paper's order or above and stay below three times its worst values.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1311_3004_gb300 import analysis, fvna
from paper_1311_3004_gb300 import workloads as wl

from helpers import Case, gpu_config, gpu_domain, oracle_params, pert_rel_linf

pytestmark = pytest.mark.gpu

P, E, R, T = fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT, fvna.BC_TAYLOR
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_3004_gb300 import build
    build.build()


def _shift_both(c, precision, plan):
    """Run `plan` = [(steps, kx, ky), ...] on the GPU and on the oracle."""
    s = fvna.Solver(gpu_config(c, precision), [gpu_domain(c)], [c.q0])
    o = oracle.Oracle(oracle_params(c), c.q0)
    for steps, kx, ky in plan:
        s.run(max_steps=steps)
        o.run(steps)
        s.shift(0, kx, ky)
        o.shift(kx, ky)
    qg, cg, sg = s.q(0), s.corner(0), s.stats(0)
    s.close()
    qo, co, so = o.q(), o.corner(), o.scalars()
    o.close()
    return qg, cg, sg, qo, co, so


PLAN = [(5, 7, -4), (4, -3, 2), (3, 0, 5), (2, -9, 0)]


@pytest.mark.parametrize("bc", [(P, P, E, R), (E, E, P, P), (R, E, E, R)])
def test_shift_parity_fp64(bc):
    nx, ny = 70, 45
    c = Case(nx, ny, wl.random_smooth(nx, ny, 2e-3, seed=11), bc=bc, delta=2e-3, x0=0.5,
             y0=-0.25)
    qg, cg, sg, qo, co, so = _shift_both(c, fvna.FP64, PLAN)
    assert np.array_equal(qg, qo)
    assert cg == co
    assert sg["steps"] == so["step"] and sg["t"] == so["t"]


def test_shift_parity_fp32():
    nx, ny = 150, 97
    c = Case(nx, ny, wl.random_smooth(nx, ny, 2e-3, seed=12), bc=(E, R, P, P), delta=2e-3)
    qg, cg, sg, qo, co, so = _shift_both(c, fvna.FP32_PERT, PLAN)
    assert pert_rel_linf(qg, qo) <= 1e-5
    assert cg == co


def test_shift_rejects_bad_arguments():
    c = Case(16, 8, wl.random_smooth(16, 8, 1e-3, seed=1))
    s = fvna.Solver(gpu_config(c), [gpu_domain(c)], [c.q0])
    L = fvna.lib()
    assert L.fvna_shift(s._h, 1, 1, 0) == fvna.ERR_ARG
    assert L.fvna_shift(s._h, 0, 16, 0) == fvna.ERR_ARG
    assert L.fvna_shift(s._h, 0, 0, -8) == fvna.ERR_ARG
    assert L.fvna_shift(s._h, 0, 0, 0) == fvna.OK
    assert L.fvna_run_moving(s._h, 1.0, 10, 0.0, 1.0, 0.0, 0, None) == fvna.ERR_ARG
    s.close()


def test_moving_taylor_parity_fp64():
    """theta_T = pi/8, window 12 x 12 units at eta = 5 moving with the shock."""
    ratio, beta, eta, angle = 1e-4, 3.5, 5, math.pi / 8
    dx, n = 1.0 / eta, 60
    q = wl.taylor_initial(n, n, dx, ratio, x0=-6.0, y0=-6.0, angle=angle)
    c = Case(n, n, q, bc=(T, T, T, T), beta=beta, delta=ratio * beta, dx=dx, x0=-6.0, y0=-6.0,
             taylor_ratio=ratio, taylor_angle=angle)
    v = (math.cos(angle), math.sin(angle))
    s = fvna.Solver(gpu_config(c), [gpu_domain(c)], [c.q0])
    sg = s.run_moving(9.0, 1.0, v, every=3)
    qg, cg = s.q(0), s.corner(0)
    s.close()
    o = oracle.Oracle(oracle_params(c), c.q0)
    oracle.run_moving(o, 9.0, 1.0, v, every=3)
    qo, co, so = o.q(), o.corner(), o.scalars()
    o.close()
    assert sg["t"] == so["t"] == 9.0 and sg["steps"] == so["step"]
    assert cg == co and cg[0] > -6.0 + 30 * dx and cg[1] > -6.0 + 10 * dx
    assert pert_rel_linf(qg, qo) <= 5e-11
    assert np.max(np.abs(qg - qo)) <= 1e-14


def _paper_table():
    tab = {}
    with open(os.path.join(GOLDEN, "taylor_shock_table_all_angles.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            k = int(f[0])
            tab[(0.0 if k == 0 else math.pi / k, f[1])] = [float(x) for x in f[2:]]
    return tab


def taylor_moving_errors(angle, eta, nu_w=0.9, t_end=100.0, ratio=1e-7, beta=3.5, side=12.0,
                         every=32):
    """E_1, E_inf of the Taylor shock at time t_end on a window that follows it
    (binary64).  theta_T = 0: a quasi-1D 30-unit window (4 rows, periodic in
    x2); otherwise a side x side window centred on the shock at t = 0."""
    dx = 1.0 / eta
    if angle == 0.0:
        nx, ny, x0, y0 = int(round(30.0 * eta)), 4, -15.0, 0.0
        bc = (T, T, P, P)
    else:
        nx = ny = int(round(side * eta))
        x0 = y0 = -0.5 * side
        bc = (T, T, T, T)
    q0 = wl.taylor_initial(nx, ny, dx, ratio, x0=x0, y0=y0, angle=angle)
    cfg = fvna.make_config(precision=fvna.FP64, beta=beta, delta=ratio * beta, dx=dx, nu_w=nu_w)
    dom = fvna.make_domain(nx, ny, bc=bc, x0=x0, y0=y0, taylor_ratio=ratio, taylor_angle=angle)
    s = fvna.Solver(cfg, [dom], [q0])
    st = s.run_moving(t_end, 0.0, (math.cos(angle), math.sin(angle)), every=every)
    q, (cx, cy) = s.q(0), s.corner(0)
    s.close()
    assert abs(st["t"] - t_end) < 1e-9 and st["status"] == 0
    e1, einf = analysis.taylor_line_errors(q, cx, cy, dx, t_end, angle, ratio)
    return e1, einf, st


@pytest.mark.parametrize("k", [0, 32, 16, 8, 4])
def test_taylor_table_on_a_moving_window(k):
    """Table tab:error-ts, nu_W = 0.9.  theta_T = 0 on a 30-unit quasi-1D
    window, eta up to 82: the paper's order and error range (within three
    times).  Rotated shocks on square windows 100 units wide (the paper ran
    its moving domains 100 wavelengths long), eta = 10, 20, 41: at least the
    paper's lowest rate (1.15), and errors at eta = 41 no worse than three
    times the paper's worst at eta = 82 (finer grids only lower them; on
    windows this wide the rotated errors are below the paper's)."""
    angle = 0.0 if k == 0 else math.pi / k
    tab = _paper_table()
    etas = [10, 20, 41, 82] if k == 0 else [10, 20, 41]
    res = [taylor_moving_errors(angle, eta, side=100.0) for eta in etas]
    e1 = np.array([r[0] for r in res])
    einf = np.array([r[1] for r in res])
    print(f"theta=pi/{k}: E1 {e1}, Einf {einf}")
    rate1 = analysis.convergence_rate(etas, e1)
    assert np.all(np.diff(e1) < 0), e1
    assert np.all(np.diff(einf) < 0), einf
    best1, worst1 = tab[(angle, "E1")][4], tab[(angle, "E1")][5]
    besti, worsti = tab[(angle, "Einf")][4], tab[(angle, "Einf")][5]
    if k == 0:
        assert rate1 > 1.5, rate1
        assert best1 / 3.0 <= e1[-1] <= 3.0 * worst1, (e1[-1], best1, worst1)
        assert besti / 3.0 <= einf[-1] <= 3.0 * worsti, (einf[-1], besti, worsti)
    else:
        assert rate1 >= 1.15, rate1
        assert e1[-1] <= 3.0 * worst1, (e1[-1], worst1)
        assert einf[-1] <= 3.0 * worsti, (einf[-1], worsti)
    for r in res:
        # the paper's CFL spread: nu never further than 1e-8 from its mean
        assert r[2]["nu_std"] < 1e-8


def test_rotated_taylor_error_is_set_by_the_window_extent():
    """The analytic values on the window's borders cut the rotated shock front
    and set its error: at theta_T = pi/8, eta = 20, a 100-unit window has an
    E_1 several times below a 12-unit one, and converges at second order
    where the 12-unit one converges at first."""
    small = [taylor_moving_errors(math.pi / 8, eta, side=12.0)[0] for eta in (10, 20)]
    wide = [taylor_moving_errors(math.pi / 8, eta, side=100.0)[0] for eta in (10, 20)]
    assert wide[1] < small[1] / 5.0, (small, wide)
    assert np.log2(small[0] / small[1]) < 1.3 and np.log2(wide[0] / wide[1]) > 1.7, (small, wide)
