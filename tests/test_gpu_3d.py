"""The 3D step on the GPU (fvna3_* through the C ABI) against the 3D CPU oracle
on the same seeded inputs: binary64 bit for bit (the kernels evaluate the
definitions in the oracle's order with no fused products), binary32
perturbation form within 1e-5 of the perturbation.  Cases cover all three
border rules on every face, ragged tile edges along every axis, the three
limiters, one-cell-thick boxes, and the full-size pulse workload's first
steps."""
import zlib

import numpy as np
import pytest

import oracle
from oracle import Params3
from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

P, E, R = fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT


def _rel(q, ref):
    amb = np.zeros_like(ref)
    amb[0] = 1.0
    return float(np.max(np.abs(q - ref)) / np.max(np.abs(ref - amb)))


def _run(nx, ny, nz, q0, bc, steps, precision=fvna.FP64, limiter=0, delta=2e-3, dx=1 / 24,
         sweeps=15, dt_fixed=0.0, tile_y=0, t_end=-np.inf, compensated=1):
    cfg = fvna.make_config(precision=precision, limiter=limiter, beta=3.5,
                           delta=delta, dx=dx, nu_w=0.8, dt_fixed=dt_fixed, tile_y=tile_y,
                           compensated=compensated)
    s = fvna.Solver3(cfg, fvna.make_domain3(nx, ny, nz, bc=bc, substeps=sweeps), q0)
    st = s.run(t_end=t_end, max_steps=steps, check=False)
    q = s.q()
    s.close()
    p = Params3(nx=nx, ny=ny, nz=nz, bc=bc, limiter=limiter, sweeps=sweeps, beta=3.5, delta=delta,
                dx=dx, nu_w=0.8, dt_fixed=dt_fixed)
    o = oracle.Oracle3(p, q0)
    o.run(steps, t_end)
    qo, so = o.q(), o.scalars()
    o.close()
    return q, st, qo, so


CASES = [
    ("extrap_ragged", (37, 29, 23), (E,) * 6, 0),
    ("periodic", (33, 34, 35), (P,) * 6, 0),
    ("reflect_mixed", (61, 19, 70), (R, E, P, P, E, R), 0),
    ("godunov", (40, 31, 17), (E, R, R, E, P, P), 1),
    ("lax_wendroff", (29, 40, 26), (P, P, E, E, R, R), 2),
    ("thin_x", (1, 40, 37), (E, E, R, E, P, P), 0),
    ("thin_z", (70, 33, 1), (R, E, E, R, E, E), 0),
    ("long_lines", (130, 140, 9), (E, E, P, P, R, R), 0),
]


@pytest.mark.parametrize("name,shape,bc,limiter", CASES, ids=[c[0] for c in CASES])
def test_3d_fp64_bit_identical_to_oracle(name, shape, bc, limiter):
    nx, ny, nz = shape
    q0 = wl.random_smooth3(nx, ny, nz, 3e-3, seed=zlib.crc32(name.encode()) % 1000)
    q, st, qo, so = _run(nx, ny, nz, q0, bc, 7, limiter=limiter)
    assert st["rc"] == fvna.OK and so["status"] == 0
    assert st["steps"] == so["step"] == 7
    assert st["t"] == so["t"]
    assert np.array_equal(q, qo), _rel(q, qo)


@pytest.mark.parametrize("name,shape,bc,limiter", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_3d_fp32_within_1e5_of_oracle(name, shape, bc, limiter):
    nx, ny, nz = shape
    q0 = wl.random_smooth3(nx, ny, nz, 3e-3, seed=zlib.crc32(name.encode()) % 1000 + 1)
    for comp in (1, 0):
        q, st, qo, so = _run(nx, ny, nz, q0, bc, 7, precision=fvna.FP32_PERT, limiter=limiter,
                             compensated=comp)
        assert st["rc"] == fvna.OK
        assert _rel(q, qo) <= 1e-5, (comp, _rel(q, qo))


@pytest.mark.parametrize("sweeps", [1, 2, 4, 8, 3, 5, 6, 7, 9, 14])
def test_3d_each_substep_alone(sweeps):
    """Every sub-step and combination of them, including an odd number of
    sub-steps (the step then ends with a copy back into the state planes)."""
    nx, ny, nz = 35, 21, 27
    q0 = wl.random_smooth3(nx, ny, nz, 3e-3, seed=sweeps)
    q, st, qo, so = _run(nx, ny, nz, q0, (E, R, P, P, R, E), 4, sweeps=sweeps, dt_fixed=0.02)
    assert st["rc"] == fvna.OK
    assert np.array_equal(q, qo), _rel(q, qo)


def test_3d_tile_heights_and_time_limit():
    """Tile heights of the x2/x3 sweeps do not change a bit; a time-limited run
    ends on t_end exactly."""
    nx, ny, nz = 45, 70, 66
    q0 = wl.random_smooth3(nx, ny, nz, 2e-3, seed=5)
    ref = None
    for ty in (4, 16, 64, 128):
        q, st, qo, so = _run(nx, ny, nz, q0, (E,) * 6, 10 ** 6, tile_y=ty, t_end=0.11)
        assert st["t"] == so["t"] == 0.11
        assert np.array_equal(q, qo)
        if ref is None:
            ref = q
        assert np.array_equal(q, ref)


def test_3d_full_size_pulse_first_steps():
    """The 256^3 pulse workload the benchmark times: the first two steps in
    binary64 match the oracle bit for bit; binary32 within 1e-5."""
    w = wl.gaussian3d(256)
    n = w["n"]
    cfg = dict(beta=w["beta"], delta=w["delta"], dx=w["dx"], nu_w=w["nu_w"])
    p = Params3(nx=n, ny=n, nz=n, bc=w["bc"], **cfg)
    qo, so = oracle.run3(p, w["q0"], 2)
    for prec, check in ((fvna.FP64, lambda q: np.array_equal(q, qo)),
                        (fvna.FP32_PERT, lambda q: _rel(q, qo) <= 1e-5)):
        s = fvna.Solver3(fvna.make_config(precision=prec, **cfg), fvna.make_domain3(n, n, n, w["bc"]),
                         w["q0"])
        st = s.run(max_steps=2)
        q = s.q()
        s.close()
        assert st["steps"] == 2
        assert check(q), _rel(q, qo)


def test_3d_nonreal_state_is_reported():
    nx = ny = nz = 12
    q0 = wl.ambient3(nx, ny, nz)
    q0[0, 5, 5, 5] = 0.3             # q1 < 1/2 at rest: non-real speeds (section 3.2)
    cfg = fvna.make_config(precision=fvna.FP64, beta=3.5, dx=0.1, nu_w=0.5)
    s = fvna.Solver3(cfg, fvna.make_domain3(nx, ny, nz), q0)
    st = s.run(max_steps=3, check=False)
    s.close()
    assert st["rc"] == fvna.ERR_NONREAL
