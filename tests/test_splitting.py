"""Pins of the oracle's Strang splitting (x1 sweep over dt/2, x2 sweep,
source, x1 sweep over dt/2) against its Godunov splitting (x1, x2, source),
on the CPU: for a linear plane wave oblique to the grid, on a fixed grid,
the splitting error of Godunov's form halves with dt (first order in time)
and Strang's falls by four (second order), with Lax-Wendroff sweeps (phi = 1,
second order in time on their own)."""
import numpy as np
import pytest

import oracle
from oracle import BC_PERIODIC, LIM_LW, LIM_MC, Params


def _wave(n, amp=1e-8):
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    k = 2 * np.pi * np.array([1.0, 2.0])          # fits the periodic unit square
    ph = k[0] * X + k[1] * Y
    kn = k / np.linalg.norm(k)
    q = np.zeros((3, n, n))
    q[0] = 1.0 + amp * np.sin(ph)
    q[1] = amp * np.sin(ph) * kn[0]               # right-going along kn
    q[2] = amp * np.sin(ph) * kn[1]
    return q, dx


def _run(n, dt, splitting, limiter, t_end=0.2):
    q0, dx = _wave(n)
    p = Params(nx=n, ny=n, bc=(BC_PERIODIC,) * 4, limiter=limiter, dx=dx, dt_fixed=dt,
               splitting=splitting, beta=3.5)
    o = oracle.Oracle(p, q0)
    o.run(10 ** 7, t_end=t_end)
    q = o.q()
    o.close()
    return q


@pytest.mark.parametrize("splitting,lo,hi", [(0, 1.7, 2.6), (1, 3.3, 4.5)])
def test_time_order_of_the_splitting(splitting, lo, hi):
    n = 64
    dx = 1.0 / n
    ref = _run(n, 0.05 * dx, splitting, LIM_LW)
    errs = [np.max(np.abs(_run(n, f * dx, splitting, LIM_LW) - ref)) for f in (0.8, 0.4, 0.2)]
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(lo <= r <= hi for r in ratios), (errs, ratios)


def test_strang_is_more_accurate_with_the_mc_limiter():
    """With the MC limiter the limiter's clipping sets the order, but the
    symmetric form still carries a smaller time error at the same dt."""
    n = 64
    dx = 1.0 / n
    e = []
    for s in (0, 1):
        ref = _run(n, 0.05 * dx, s, LIM_MC)
        e.append(np.max(np.abs(_run(n, 0.8 * dx, s, LIM_MC) - ref)))
    assert e[1] < 0.6 * e[0], e


def test_strang_without_the_x1_sweep_is_godunov():
    """With the x1 sweep switched off both forms are the same step, bit for bit."""
    n = 32
    q0, dx = _wave(n, 1e-4)
    res = []
    for s in (0, 1):
        p = Params(nx=n, ny=n, bc=(BC_PERIODIC,) * 4, dx=dx, nu_w=0.9, splitting=s, sweeps=6,
                   delta=1e-3)
        o = oracle.Oracle(p, q0)
        o.run(20)
        res.append(o.q())
        o.close()
    assert np.array_equal(res[0], res[1])


def test_strang_reduces_the_rotated_taylor_shock_error():
    """Section 4.1's Taylor shock at theta_T = pi/32 and pi/8 (eta = 10, moving
    12 x 12 window to t = 30): the symmetric order of the fractional steps
    lowers E_1 and E_inf, i.e. the angle dependence the paper reports."""
    import math
    from oracle import BC_TAYLOR
    from paper_1311_3004_gb300 import analysis
    from paper_1311_3004_gb300 import workloads as wl
    ratio, beta, eta, side, t_end = 1e-7, 3.5, 10, 12.0, 30.0
    for k in (32, 8):
        angle, dx, n = math.pi / k, 1.0 / eta, int(side * eta)
        e = []
        for s in (0, 1):
            q0 = wl.taylor_initial(n, n, dx, ratio, x0=-6.0, y0=-6.0, angle=angle)
            p = Params(nx=n, ny=n, bc=(BC_TAYLOR,) * 4, beta=beta, delta=ratio * beta, dx=dx,
                       nu_w=0.9, x0=-6.0, y0=-6.0, taylor_ratio=ratio, taylor_angle=angle,
                       splitting=s)
            o = oracle.Oracle(p, q0)
            oracle.run_moving(o, t_end, 0.0, (math.cos(angle), math.sin(angle)), every=32)
            cx, cy = o.corner()
            e.append(analysis.taylor_line_errors(o.q(), cx, cy, dx, t_end, angle, ratio))
            o.close()
        assert e[1][0] < 0.7 * e[0][0] and e[1][1] < 0.7 * e[0][1], (k, e)
