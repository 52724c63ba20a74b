"""Pins of the oracle's moving domain (section 4: in the second stage of a run
the domain moves with the wave), on the CPU.

- A shift of a doubly periodic window is a cyclic roll of the state, and the
  corner moves by whole cells.
- Cells entering through an extrapolation border copy the nearest old cell.
- A plane Taylor shock (eq. OurTaylorS) in a 2D window, periodic across the
  propagation direction and moved along both axes, is row for row the
  quasi-1D moving run.
- With the window following the theta_T = 0 shock, the errors of section 4.1
  match those of a long static domain.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import BC_EXTRAP, BC_PERIODIC, BC_TAYLOR, Params
from paper_1311_3004_gb300 import workloads as wl


def test_periodic_shift_is_a_roll():
    nx, ny, dx = 23, 17, 0.1
    q0 = wl.random_smooth(nx, ny, 1e-3, seed=7)
    p = Params(nx=nx, ny=ny, bc=(BC_PERIODIC,) * 4, dx=dx, x0=0.25, y0=-1.5)
    o = oracle.Oracle(p, q0)
    o.shift(5, -3)
    q = o.q()
    ref = np.roll(q0, shift=(3, -5), axis=(1, 2))
    assert np.array_equal(q, ref)
    assert o.corner() == (0.25 + 5 * dx, -1.5 + (-3) * dx)
    o.shift(-5, 3)
    assert np.array_equal(o.q(), q0)
    with pytest.raises(ValueError):
        o.shift(nx, 0)
    o.close()


def test_extrapolation_shift_copies_the_edge():
    nx, ny = 12, 9
    q0 = wl.random_smooth(nx, ny, 1e-3, seed=3)
    p = Params(nx=nx, ny=ny, bc=(BC_EXTRAP,) * 4, dx=0.5)
    o = oracle.Oracle(p, q0)
    o.shift(4, 2)
    q = o.q()
    # cells with an old counterpart moved; new ones copy the nearest old cell
    assert np.array_equal(q[:, :ny - 2, :nx - 4], q0[:, 2:, 4:])
    for j in range(ny):
        for i in range(nx):
            si, sj = min(i + 4, nx - 1), min(j + 2, ny - 1)
            assert np.array_equal(q[:, j, i], q0[:, sj, si])
    o.close()


def test_diagonal_move_of_a_plane_shock_is_row_for_row_the_1d_run():
    """theta_T = 0 shock in a 2D window, periodic in x2, moved along both axes
    (velocity (1, 0.37)): every x2 shift is a roll of identical rows, so every
    row equals the quasi-1D moving run bit for bit, and the corner follows the
    rounded displacement."""
    eta, ratio, beta, T, t1 = 5, 1e-7, 3.5, 20.0, 2.0
    dx, x0 = 1.0 / eta, -10.0
    nx = int(round(20.0 * eta))
    res = []
    for ny, vy, bcy in ((1, 0.0, BC_EXTRAP), (9, 0.37, BC_PERIODIC)):
        q0 = wl.taylor_initial(nx, ny, dx, ratio, x0=x0, y0=1.0)
        p = Params(nx=nx, ny=ny, bc=(BC_TAYLOR, BC_TAYLOR, bcy, bcy), beta=beta,
                   delta=ratio * beta, dx=dx, nu_w=0.9, x0=x0, y0=1.0, taylor_ratio=ratio)
        o = oracle.Oracle(p, q0)
        oracle.run_moving(o, T, t1, (1.0, vy), every=5)
        sc = o.scalars()
        assert sc["t"] == T and sc["status"] == 0
        res.append((o.q(), o.corner(), sc))
        o.close()
    (q1d, c1d, s1d), (q2d, c2d, s2d) = res
    for j in range(q2d.shape[1]):
        assert np.array_equal(q2d[:, j, :], q1d[:, 0, :]), j
    assert c2d[0] == c1d[0] and s2d["step"] == s1d["step"]
    kx = round((c1d[0] - x0) / dx)
    ky = round((c2d[1] - 1.0) / dx)
    assert kx == math.floor(1.0 * (T - t1) / dx + 0.5) or abs(kx * dx - (T - t1)) <= dx
    assert ky == math.floor(0.37 * (T - t1) / dx + 0.5)
    assert kx > 50 and ky > 20


def _taylor_errors_line(q, dx, x0, T, ratio=1e-7):
    x = x0 + (np.arange(q.shape[2]) + 0.5) * dx
    sel = np.abs(x - T) <= 5.0
    num = q[0, 0, sel] - 1.0
    ref = -ratio * np.tanh(x[sel] - T)
    return (np.sum(np.abs(num - ref)) / np.sum(np.abs(ref)),
            np.max(np.abs(num - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("eta", [5, 10])
def test_moving_window_keeps_the_taylor_shock_errors(eta):
    """theta_T = 0: a 30-unit window that follows the shock to t = 100 gives the
    errors of section 4.1 that a static 140-unit domain gives."""
    ratio, beta, T, dx = 1e-7, 3.5, 100.0, 1.0 / eta
    res = []
    for x0, length, moving in ((-15.0, 30.0, True), (-20.0, 140.0, False)):
        nx = int(round(length * eta))
        q0 = wl.taylor_initial(nx, 1, dx, ratio, x0=x0)
        p = Params(nx=nx, ny=1, bc=(BC_TAYLOR, BC_TAYLOR, BC_EXTRAP, BC_EXTRAP), beta=beta,
                   delta=ratio * beta, dx=dx, nu_w=0.9, x0=x0, taylor_ratio=ratio)
        o = oracle.Oracle(p, q0)
        if moving:
            oracle.run_moving(o, T, 0.0, (1.0, 0.0), every=8)
        else:
            o.run(10 ** 8, t_end=T)
        assert abs(o.scalars()["t"] - T) < 1e-12
        res.append(_taylor_errors_line(o.q(), dx, o.corner()[0], T, ratio))
        o.close()
    (e1m, eim), (e1s, eis) = res
    assert abs(e1m - e1s) <= 0.02 * e1s, (e1m, e1s)
    assert abs(eim - eis) <= 0.02 * eis, (eim, eis)


def test_set_bc_takes_effect_from_the_next_step():
    """A border rule changed before the first step gives the run of a domain
    created with that rule, bit for bit; changing it mid-run changes the
    result only from then on."""
    nx, ny = 30, 20
    q0 = wl.random_smooth(nx, ny, 1e-3, seed=5)
    base = dict(nx=nx, ny=ny, dx=0.1, delta=1e-3)
    o1 = oracle.Oracle(Params(bc=(BC_EXTRAP,) * 4, **base), q0)
    o2 = oracle.Oracle(Params(bc=(oracle.BC_REFLECT, BC_EXTRAP, BC_EXTRAP, BC_EXTRAP), **base), q0)
    o2.set_bc(0, BC_EXTRAP)
    o1.run(15)
    o2.run(15)
    assert np.array_equal(o1.q(), o2.q())
    o3 = oracle.Oracle(Params(bc=(BC_EXTRAP,) * 4, **base), q0)
    o3.run(5)
    o3.set_bc(1, oracle.BC_REFLECT)
    o3.run(10)
    assert not np.array_equal(o3.q(), o1.q())
    for o in (o1, o2, o3):
        o.close()
