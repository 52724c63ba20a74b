"""Pins of the three-dimensional CPU oracle (oracle/fvna_oracle3d.c) against
what the paper and the mathematics fix, independently of the oracle itself:
the Roe condition of section 3.2 for the flux of eq. adim:q with a third
velocity component, consistency with the flux Jacobian, exact reduction to
the (pinned) 2D oracle for states that do not vary along one axis, discrete
conservation with periodic borders, mirror symmetry, the linear oblique plane
wave and the linear spherical wave (closed forms, with convergence)."""
import numpy as np
import pytest

import oracle
from oracle import Params, Params3, BC_PERIODIC, BC_EXTRAP, BC_REFLECT, LIM_MC, LIM_LW
from paper_1311_3004_gb300 import workloads as wl


def flux3_x1(q, beta):
    """f_1 of eq. adim:q with three velocity components:
    q2/(q1)^2 ((q1)^2, q2, q3, q4) + phi (0, 1, 0, 0)."""
    q1, q2, q3, q4 = q
    phi = q1 + (beta - 1.0) * (q1 - 1.0) ** 2
    return np.array([q2, q2 * q2 / q1 ** 2 + phi, q2 * q3 / q1 ** 2, q2 * q4 / q1 ** 2])


def _pairs(rng, n, scale):
    qL = np.zeros((n, 4))
    qR = np.zeros((n, 4))
    for q in (qL, qR):
        q[:, 0] = 1.0 + scale * rng.uniform(-1, 1, n)
        q[:, 1:] = scale * rng.uniform(-1, 1, (n, 3))
    return qL, qR


@pytest.mark.parametrize("scale", [1e-4, 3e-2, 0.2])
def test_roe_condition_and_wave_sum_3d(scale):
    """sum_p s_p W_p = f(Q_R) - f(Q_L) (eq. RoeCond) and sum_p W_p = dQ."""
    rng = np.random.default_rng(31)
    beta = 3.5
    for qL, qR in zip(*_pairs(rng, 200, scale)):
        s, W, am, ap, nr = oracle.interface3(beta, qL, qR)
        assert not nr
        df = flux3_x1(qR, beta) - flux3_x1(qL, beta)
        ref = max(np.max(np.abs(df)), 1e-300)
        tol = 1e-14 + 1e-13 * ref          # the flux itself is of order one
        assert np.max(np.abs(s @ W - df)) <= tol, (s @ W, df)
        assert np.allclose(W.sum(axis=0), qR - qL, rtol=0, atol=1e-15)
        assert np.max(np.abs(am + ap - df)) <= tol
        # the transverse families carry only their own component
        assert W[2, [0, 1, 3]].tolist() == [0.0, 0.0, 0.0]
        assert W[3, [0, 1, 2]].tolist() == [0.0, 0.0, 0.0]
        assert s[2] == s[3]


def test_roe_speeds_tend_to_jacobian_eigenvalues():
    """Consistency: as Q_R -> Q_L the speeds tend to the eigenvalues of df/dq
    (finite differences of the flux), u + c, u - c and u twice."""
    beta = 4.8
    q = np.array([1.02, 0.03, -0.015, 0.02])
    h = 1e-7
    J = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        J[:, k] = (flux3_x1(q + e, beta) - flux3_x1(q - e, beta)) / (2 * h)
    ev = np.sort(np.linalg.eigvals(J).real)
    s, *_ = oracle.interface3(beta, q, q * (1 + 1e-12))
    assert np.allclose(np.sort(s), ev, atol=1e-6), (s, ev)


def _random3(nx, ny, nz, amp, seed, q4=True):
    rng = np.random.default_rng(seed)
    X, Y, Z = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny, np.arange(nz) / nz,
                          indexing="xy")
    X, Y, Z = (a.transpose(2, 0, 1) for a in (X, Y, Z))     # (nz, ny, nx)
    q = np.zeros((4, nz, ny, nx))
    q[0] = 1.0
    for f in range(4 if q4 else 3):
        for _ in range(4):
            kx, ky, kz = rng.integers(0, 3, size=3)
            q[f] += amp * rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y + kz * Z) +
                                                      rng.uniform(0, 2 * np.pi)) / 4
    return q


@pytest.mark.parametrize("bcz", [BC_PERIODIC, BC_EXTRAP, BC_REFLECT])
def test_x3_invariant_state_equals_the_2d_scheme(bcz):
    """A state that does not vary along x3 and has no x3 momentum takes, in
    three dimensions, exactly the 2D oracle's step: the x3 sweep sees no jump
    and the third Laplacian term vanishes (fixed dt, all borders)."""
    nx, ny, nz, steps = 23, 17, 4, 6
    q2d = wl.random_smooth(nx, ny, 3e-3, seed=33)
    bc2 = (BC_PERIODIC, BC_PERIODIC, BC_EXTRAP, BC_REFLECT)
    p2 = Params(nx=nx, ny=ny, bc=bc2, beta=3.5, delta=2e-3, dx=1 / 16, dt_fixed=0.04)
    q2, _ = oracle.run(p2, q2d, steps)
    q3d = np.zeros((4, nz, ny, nx))
    q3d[:3] = q2d[:, None]
    p3 = Params3(nx=nx, ny=ny, nz=nz, bc=bc2 + (bcz, bcz), beta=3.5, delta=2e-3, dx=1 / 16,
                 dt_fixed=0.04)
    q3, sc = oracle.run3(p3, q3d, steps)
    assert sc["step"] == steps
    for k in range(nz):
        assert np.array_equal(q3[:3, k], q2)
    assert np.all(q3[3] == 0.0)


def test_x2_invariant_state_equals_the_2d_scheme_in_x1_x3():
    """Rotated: a state that does not vary along x2 and has no x2 momentum is
    the 2D scheme in the (x1, x3) plane, with (q2, q4) of the 3D state in the
    place of (q2, q3) (sweeps bit for bit; the source to rounding, its three
    Laplacian terms being summed in another order)."""
    nx, ny, nz, steps = 19, 3, 21, 5
    q2d = wl.random_smooth(nx, nz, 3e-3, seed=34)
    bc2 = (BC_EXTRAP, BC_EXTRAP, BC_REFLECT, BC_EXTRAP)
    q3d = np.zeros((4, nz, ny, nx))
    q3d[0] = q2d[0][:, None, :]
    q3d[1] = q2d[1][:, None, :]
    q3d[3] = q2d[2][:, None, :]
    for delta, sweeps2, sweeps3, tol in ((0.0, 3, 7, 0.0), (2e-3, 7, 15, 1e-15)):
        p2 = Params(nx=nx, ny=nz, bc=bc2, beta=3.5, delta=delta, dx=1 / 16, dt_fixed=0.04,
                    sweeps=sweeps2)
        q2, _ = oracle.run(p2, q2d, steps)
        p3 = Params3(nx=nx, ny=ny, nz=nz, bc=(bc2[0], bc2[1], BC_PERIODIC, BC_PERIODIC,
                                               bc2[2], bc2[3]),
                     beta=3.5, delta=delta, dx=1 / 16, dt_fixed=0.04, sweeps=sweeps3)
        q3, _ = oracle.run3(p3, q3d, steps)
        for j in range(ny):
            got = np.stack([q3[0, :, j], q3[1, :, j], q3[3, :, j]])
            err = np.max(np.abs(got - q2))
            assert err <= tol, (delta, err)
        assert np.all(q3[2] == 0.0)


def test_periodic_conservation_3d():
    """Periodic borders: the flux differences telescope and the Laplacian sums
    to zero, so every field's sum is conserved to rounding."""
    n = 14
    q0 = _random3(n, n, n, 4e-3, seed=35)
    p = Params3(nx=n, ny=n, nz=n, bc=(BC_PERIODIC,) * 6, beta=3.5, delta=3e-3, dx=1 / 16)
    q, sc = oracle.run3(p, q0, 40)
    assert sc["status"] == 0 and sc["step"] == 40
    for f in range(4):
        d = abs(q[f].sum() - q0[f].sum())
        assert d <= 2e-13 * max(1.0, np.abs(q0[f]).sum() / q0[f].size) * q0[f].size ** 0.5, (f, d)
    assert np.max(np.abs(q - q0)) > 1e-5          # something happened


def test_mirror_symmetry_3d():
    """A pulse centred in the box stays mirror-symmetric about each mid-plane
    (the normal momentum odd, the rest even)."""
    n = 16
    c = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    q0 = np.zeros((4, n, n, n))
    q0[0] = 1.0 + 2e-3 * np.exp(-(X * X + Y * Y + Z * Z) / (2 * 0.12 ** 2))
    p = Params3(nx=n, ny=n, nz=n, bc=(BC_EXTRAP,) * 6, beta=3.5, delta=1e-3, dx=1 / n)
    q, _ = oracle.run3(p, q0, 12)
    for ax, f in ((3, 1), (2, 2), (1, 3)):
        m = np.flip(q, axis=ax)
        for k in range(4):
            sign = -1.0 if k == f else 1.0
            assert np.max(np.abs(q[k] - sign * m[k])) <= 1e-16, (ax, k)


def _oblique_error(n, limiter):
    """Linear plane wave along (1, 2, 2)/3 in a periodic unit cube, no
    dissipation: q1 - 1 = A sin(k.x - |k| t), momentum (q1 - 1) k/|k|."""
    A, T = 1e-8, 0.2
    kv = 2 * np.pi * np.array([1.0, 2.0, 2.0])
    nv = kv / np.linalg.norm(kv)
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    ph = kv[0] * X + kv[1] * Y + kv[2] * Z
    q0 = np.zeros((4, n, n, n))
    w = A * np.sin(ph)
    q0[0] = 1.0 + w
    for k in range(3):
        q0[1 + k] = w * nv[k]
    p = Params3(nx=n, ny=n, nz=n, bc=(BC_PERIODIC,) * 6, beta=3.5, dx=1.0 / n, nu_w=0.8,
                limiter=limiter)
    q, sc = oracle.run3(p, q0, 10 ** 6, t_end=T)
    assert sc["t"] == T
    exact = A * np.sin(ph - np.linalg.norm(kv) * T)
    return np.mean(np.abs(q[0] - 1.0 - exact)) / np.mean(np.abs(exact))


def test_oblique_plane_wave_3d():
    """The oblique wave moves at the unit sound speed along its direction in
    all three sweeps together; the L1 error falls with the mesh at close to
    second order with the Lax-Wendroff correction and better than first order
    with MC."""
    e1, e2 = _oblique_error(24, LIM_LW), _oblique_error(48, LIM_LW)
    assert e2 < 0.05, e2
    assert np.log2(e1 / e2) > 1.7, (e1, e2)
    m1, m2 = _oblique_error(24, LIM_MC), _oblique_error(48, LIM_MC)
    assert np.log2(m1 / m2) > 1.2, (m1, m2)


def _spherical_error_3d(n_per_unit):
    """Linear spherical pulse at the corner of the octant x, y, z > 0 with
    reflective walls on the three low faces (the mirror images complete the
    sphere): p(R, 0) = g(R), u = 0 gives p(R, t) = [(R - t) g(R - t) +
    (R + t) g(R + t)] / (2R)."""
    amp, sig, T, L = 1e-8, 0.15, 0.6, 1.5
    n = int(L * n_per_unit)
    c = (np.arange(n) + 0.5) / n_per_unit
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(X * X + Y * Y + Z * Z)
    g = lambda x: amp * np.exp(-x * x / (2 * sig * sig))
    q0 = np.zeros((4, n, n, n))
    q0[0] = 1.0 + g(R)
    p = Params3(nx=n, ny=n, nz=n, bc=(BC_REFLECT, BC_EXTRAP) * 3, beta=3.5, dx=1.0 / n_per_unit,
                nu_w=0.8)
    q, sc = oracle.run3(p, q0, 10 ** 6, t_end=T)
    exact = ((R - T) * g(R - T) + (R + T) * g(R + T)) / (2 * R)
    return np.sum(np.abs(q[0] - 1.0 - exact)) / np.sum(np.abs(exact))


def test_linear_spherical_wave_3d():
    """The 3D Cartesian scheme spreads a pulse spherically (no axisymmetric
    reduction, no geometric source): the error against the closed form is
    small and falls at better than first order."""
    e1, e2 = _spherical_error_3d(20), _spherical_error_3d(40)
    assert e2 < 0.05, (e1, e2)
    assert np.log2(e1 / e2) > 1.3, (e1, e2)
