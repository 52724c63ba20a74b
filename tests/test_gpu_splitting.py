"""Strang splitting on the GPU (x1 sweep over dt/2, x2 sweep with the source,
x1 sweep over dt/2, the result copied back), through the C ABI, against the
oracle's Strang step: bit for bit in binary64 away from driven borders,
within the binary32 bar otherwise; with several domains and many steps (the
tile counters of the binary32 sweeps are reset by the copy that ends a step);
and the rotated Taylor shock of section 4.1, whose error Strang's order
lowers at every resolution."""
import math

import numpy as np
import pytest

import oracle
from paper_1311_3004_gb300 import analysis, fvna
from paper_1311_3004_gb300 import workloads as wl

from helpers import Case, gpu_domain, oracle_params, pert_rel_linf

pytestmark = pytest.mark.gpu

P, E, R, T = fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT, fvna.BC_TAYLOR


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_3004_gb300 import build
    build.build()


def _cfg(c, precision):
    return fvna.make_config(precision=precision, limiter=c.limiter, beta=c.beta, delta=c.delta,
                            dx=c.dx, nu_w=c.nu_w, splitting=fvna.SPLIT_STRANG)


def _oracle(c, steps):
    p = oracle_params(c)
    p.splitting = 1
    return oracle.run(p, c.q0, steps)


@pytest.mark.parametrize("bc", [(P, P, E, R), (E, R, P, P)])
def test_strang_fp64_bit_identical(bc):
    nx, ny = 97, 66
    c = Case(nx, ny, wl.random_smooth(nx, ny, 2e-3, seed=21), bc=bc, delta=2e-3)
    s = fvna.Solver(_cfg(c, fvna.FP64), [gpu_domain(c)], [c.q0])
    st = s.run(max_steps=25)
    qg = s.q(0)
    s.close()
    qo, so = _oracle(c, 25)
    assert np.array_equal(qg, qo)
    assert st["t"] == so["t"] and st["steps"] == so["step"]


def test_strang_fp64_timed_steps_equal_graph_steps():
    nx, ny = 64, 48
    c = Case(nx, ny, wl.random_smooth(nx, ny, 2e-3, seed=22), bc=(E, E, P, P), delta=2e-3)
    s1 = fvna.Solver(_cfg(c, fvna.FP64), [gpu_domain(c)], [c.q0])
    for _ in range(6):
        s1.step_timed()
    s2 = fvna.Solver(_cfg(c, fvna.FP64), [gpu_domain(c)], [c.q0])
    s2.run(max_steps=6)
    assert np.array_equal(s1.q(0), s2.q(0))
    s1.close()
    s2.close()


def test_strang_fp32_against_oracle_many_domains():
    doms, q0s, cases = [], [], []
    for k, (nx, ny) in enumerate([(150, 97), (64, 200), (131, 70)]):
        c = Case(nx, ny, wl.random_smooth(nx, ny, 2e-3, seed=30 + k), bc=(E, E, E, R),
                 delta=2e-3)
        cases.append(c)
        doms.append(gpu_domain(c))
        q0s.append(c.q0)
    s = fvna.Solver(_cfg(cases[0], fvna.FP32_PERT), doms, q0s)
    s.run(max_steps=30)
    for k, c in enumerate(cases):
        qo, _ = _oracle(c, 30)
        assert pert_rel_linf(s.q(k), qo) <= 1e-5, k
    s.close()


def test_strang_driven_border_parity():
    ratio, beta, n, dx = 1e-4, 3.5, 60, 1.0 / 10
    q = wl.taylor_initial(n, n, dx, ratio, x0=-3.0, y0=-3.0, angle=math.pi / 8)
    c = Case(n, n, q, bc=(T, T, T, T), beta=beta, delta=ratio * beta, dx=dx, x0=-3.0, y0=-3.0,
             taylor_ratio=ratio, taylor_angle=math.pi / 8)
    s = fvna.Solver(_cfg(c, fvna.FP64), [gpu_domain(c)], [c.q0])
    s.run(max_steps=40)
    qg = s.q(0)
    s.close()
    qo, _ = _oracle(c, 40)
    assert pert_rel_linf(qg, qo) <= 5e-11
    assert np.max(np.abs(qg - qo)) <= 1e-14


def test_strang_lowers_the_rotated_taylor_error():
    """theta_T = pi/8, t = 100, eta = 10, 20, 41 (binary64, moving 12 x 12
    window): E_1 with Strang's order below E_1 with Godunov's at every eta."""
    ratio, beta, angle = 1e-7, 3.5, math.pi / 8
    for eta in (10, 20, 41):
        dx, n = 1.0 / eta, int(12 * eta)
        q0 = wl.taylor_initial(n, n, dx, ratio, x0=-6.0, y0=-6.0, angle=angle)
        e = []
        for split in (fvna.SPLIT_GODUNOV, fvna.SPLIT_STRANG):
            cfg = fvna.make_config(precision=fvna.FP64, beta=beta, delta=ratio * beta, dx=dx,
                                   nu_w=0.9, splitting=split)
            dom = fvna.make_domain(n, n, bc=(T,) * 4, x0=-6.0, y0=-6.0, taylor_ratio=ratio,
                                   taylor_angle=angle)
            s = fvna.Solver(cfg, [dom], [q0])
            s.run_moving(100.0, 0.0, (math.cos(angle), math.sin(angle)), every=32)
            cx, cy = s.corner(0)
            e.append(analysis.taylor_line_errors(s.q(0), cx, cy, dx, 100.0, angle, ratio)[0])
            s.close()
        print(f"eta={eta}: E1 Godunov {e[0]:.3e}, Strang {e[1]:.3e}")
        assert e[1] < e[0], (eta, e)
