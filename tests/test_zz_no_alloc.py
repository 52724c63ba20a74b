"""fvna_step_noalloc: the binary64 step for callers that cannot allocate device
memory at run time (they hand over their own input and output buffers; the
library's intermediate planes live in a fixed device array).  Checked against
the regular entry points, which allocate, on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12   # perturbation-relative L_inf, the binary64 bar of the other GPU tests


def _rel(a, ref):
    amb = np.zeros_like(ref)
    amb[0] = 1.0
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref - amb)))


def test_noalloc_step_matches_regular_step_twice():
    torch = pytest.importorskip("torch")
    from paper_1311_3004_gb300 import build
    build.build()
    nx, ny, dt = 150, 97, 0.012
    bc = (fvna.BC_PERIODIC, fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT)
    q0 = wl.random_smooth(nx, ny, 2e-3, seed=61)
    cfg = fvna.make_config(precision=fvna.FP64, beta=3.5, delta=2e-3, dx=1.0 / 32, dt_fixed=dt)
    dom = fvna.make_domain(nx, ny, bc=bc)

    # regular entry points (they allocate): two steps with the same dt
    s = fvna.Solver(cfg, [dom], [q0])
    s.run(max_steps=1)
    ref1 = s.q(0)
    s.run(max_steps=1)
    ref2 = s.q(0)
    s.close()

    # the allocation-free step, caller-owned buffers, two calls in a row
    qa = torch.from_numpy(q0).cuda()
    qb = torch.empty_like(qa)
    rc, smax1 = fvna.step_noalloc(cfg, dom, qa, qb, 0.0, dt)
    assert rc == fvna.OK
    got1 = qb.cpu().numpy()
    rc, smax2 = fvna.step_noalloc(cfg, dom, qb, qa, dt, dt)
    assert rc == fvna.OK
    got2 = qa.cpu().numpy()
    assert _rel(got1, ref1) <= TOL
    assert _rel(got2, ref2) <= TOL
    assert 0.9 < smax1 < 1.1 and 0.9 < smax2 < 1.1

    # in place (q_out == q_in) gives the same result
    qc = torch.from_numpy(q0).cuda()
    assert fvna.step_noalloc(cfg, dom, qc, qc, 0.0, dt)[0] == fvna.OK
    assert _rel(qc.cpu().numpy(), ref1) <= TOL


def test_noalloc_rejects_domains_beyond_its_fixed_size():
    torch = pytest.importorskip("torch")
    n = int(np.sqrt(fvna.NOALLOC_MAX_CELLS)) + 8
    cfg = fvna.make_config(precision=fvna.FP64, dx=0.01, dt_fixed=0.001)
    dom = fvna.make_domain(n, n)
    q = torch.zeros((3, 1, 1), dtype=torch.float64, device="cuda")
    rc, _ = fvna.step_noalloc(cfg, dom, q, q, 0.0, 0.001)
    assert rc == fvna.ERR_SIZE
    bad = fvna.make_config(precision=fvna.FP32_PERT, dx=0.01)
    assert fvna.step_noalloc(bad, fvna.make_domain(8, 8), q, q, 0.0, 0.001)[0] == fvna.ERR_ARG
