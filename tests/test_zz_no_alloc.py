"""fvna_step_noalloc: the binary64 step for callers that cannot allocate device
memory at run time (they hand over their own input and output buffers; the
library's intermediate planes live in a fixed device array).  Checked against
the regular entry points, which allocate, on two calls in a row: the same
kernels run on the same values, so the results must agree bit for bit.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _two_steps_both_ways(cfg, dom, q0, t0, dt):
    """Two steps of the regular context and two allocation-free calls in a row
    (plus one in place); returns the pairs of states and the two max|s|."""
    torch = pytest.importorskip("torch")
    from paper_1311_3004_gb300 import build
    build.build()
    s = fvna.Solver(cfg, [dom], [q0])
    s.run(max_steps=1)
    ref1 = s.q(0)
    s.run(max_steps=1)
    ref2 = s.q(0)
    s.close()

    qa = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    qb = torch.empty_like(qa)
    rc, smax1 = fvna.step_noalloc(cfg, dom, qa, qb, t0, dt)
    assert rc == fvna.OK, fvna.strerror(rc)
    got1 = qb.cpu().numpy()
    rc, smax2 = fvna.step_noalloc(cfg, dom, qb, qa, t0 + dt, dt)
    assert rc == fvna.OK, fvna.strerror(rc)
    got2 = qa.cpu().numpy()
    qc = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    assert fvna.step_noalloc(cfg, dom, qc, qc, t0, dt)[0] == fvna.OK
    return (got1, ref1), (got2, ref2), qc.cpu().numpy(), (smax1, smax2)


def test_noalloc_step_matches_regular_step_twice():
    nx, ny, dt = 150, 97, 0.012
    bc = (fvna.BC_PERIODIC, fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT)
    q0 = wl.random_smooth(nx, ny, 2e-3, seed=61)
    cfg = fvna.make_config(precision=fvna.FP64, beta=3.5, delta=2e-3, dx=1.0 / 32, dt_fixed=dt)
    dom = fvna.make_domain(nx, ny, bc=bc)
    (g1, r1), (g2, r2), inplace, (s1, s2) = _two_steps_both_ways(cfg, dom, q0, 0.0, dt)
    assert np.array_equal(g1, r1)
    assert np.array_equal(g2, r2)
    assert np.array_equal(inplace, r1)
    assert 0.9 < s1 < 1.1 and 0.9 < s2 < 1.1


def test_noalloc_axisymmetric_focused_drive():
    """The (z, r) form with the focused drive on the z = 0 border (the drive is
    evaluated inside the sweep here, from a precomputed buffer in the regular
    context: the same device function on the same arguments)."""
    nz, nr, dx = 120, 64, 1.0 / 20
    cfg = fvna.make_config(precision=fvna.FP64, geometry=fvna.AXISYMMETRIC, beta=3.5,
                           delta=1e-3, dx=dx, dt_fixed=0.4 * dx)
    dom = fvna.make_domain(nz, nr, bc=(fvna.BC_HIFU, fvna.BC_EXTRAP, fvna.BC_REFLECT,
                                       fvna.BC_EXTRAP),
                           envelope=0, t0=6.3, amp=2e-4, focal=4.0, aperture=2.0)
    q0 = wl.random_smooth(nz, nr, 1e-4, seed=62)
    (g1, r1), (g2, r2), inplace, _ = _two_steps_both_ways(cfg, dom, q0, 6.3, 0.4 * dx)
    assert np.abs(r2[0, :, 0] - 1.0).max() > 1e-5   # the drive reached the first column
    assert np.array_equal(g1, r1)
    assert np.array_equal(g2, r2)
    assert np.array_equal(inplace, r1)


def test_noalloc_taylor_borders():
    """Analytic Taylor-shock values (eq. OurTaylorS, rotated) on every border."""
    n, eta, ang = 96, 12.0, np.pi / 8
    dx = 1.0 / eta
    ratio = 1e-3
    x0 = y0 = -n * dx / 2
    xc = x0 + (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc)
    q1 = 1.0 - ratio * np.tanh(X * np.cos(ang) + Y * np.sin(ang))
    q0 = np.stack([q1, (q1 - 1.0) * np.cos(ang), (q1 - 1.0) * np.sin(ang)])
    cfg = fvna.make_config(precision=fvna.FP64, beta=3.5, delta=3.5 * ratio, dx=dx,
                           dt_fixed=0.8 * dx)
    dom = fvna.make_domain(n, n, bc=(fvna.BC_TAYLOR,) * 4, x0=x0, y0=y0, taylor_ratio=ratio,
                           taylor_angle=ang)
    (g1, r1), (g2, r2), inplace, _ = _two_steps_both_ways(cfg, dom, q0, 0.0, 0.8 * dx)
    assert np.array_equal(g1, r1)
    assert np.array_equal(g2, r2)
    assert np.array_equal(inplace, r1)


def test_noalloc_rejects_domains_beyond_its_fixed_size():
    torch = pytest.importorskip("torch")
    L = fvna.lib()
    n = int(np.sqrt(fvna.NOALLOC_MAX_CELLS)) + 8
    q = torch.zeros((3, 1, 1), dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(q.data_ptr())
    call = lambda cfg, dom: L.fvna_step_noalloc(ctypes.byref(cfg), ctypes.byref(dom), p, p,
                                                0.0, 0.001, None, None)
    cfg = fvna.make_config(precision=fvna.FP64, dx=0.01, dt_fixed=0.001)
    # the size is refused before any buffer is touched
    assert call(cfg, fvna.make_domain(n, n)) == fvna.ERR_SIZE
    assert call(fvna.make_config(precision=fvna.FP32_PERT, dx=0.01),
                fvna.make_domain(8, 8)) == fvna.ERR_ARG
    # the checks fvna_init makes
    assert call(fvna.make_config(precision=fvna.FP64, dx=float("inf")),
                fvna.make_domain(8, 8)) == fvna.ERR_ARG
    assert call(cfg, fvna.make_domain(8, 8, bc=(fvna.BC_HIFU,) + (fvna.BC_EXTRAP,) * 3,
                                      focal=0.0)) == fvna.ERR_ARG
