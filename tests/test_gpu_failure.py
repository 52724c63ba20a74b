"""Failure detection on the GPU without faulting it: a bounded wait that runs
out.  The binary32 sweeps wait on an mbarrier for each tile their TMA copies
bring in; `wait_limit < 0` makes every such first wait give up before its
first poll.  The kernel then records the timeout, waits (with the default
limit) for the copy in flight to land, and returns; the host reads
FVNA_ERR_TIMEOUT and the context stays usable."""
import numpy as np
import pytest

from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

from helpers import Case, pert_rel_linf, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _case():
    return Case(nx=300, ny=200, q0=wl.random_smooth(300, 200, 1e-3, seed=9),
                bc=(fvna.BC_EXTRAP,) * 4, delta=1e-3)


def test_wait_timeout_is_reported_and_the_context_stays_usable():
    c = _case()
    cfg = fvna.make_config(precision=fvna.FP32_PERT, beta=c.beta, delta=c.delta, dx=c.dx,
                           nu_w=c.nu_w, wait_limit=-1)
    s = fvna.Solver(cfg, [fvna.make_domain(c.nx, c.ny, bc=c.bc)], [c.q0])
    st = s.run(max_steps=3, check=False)
    assert st["rc"] == fvna.ERR_TIMEOUT, fvna.strerror(st["rc"])
    assert st["status"] == fvna.ERR_TIMEOUT
    assert st["steps"] == 1          # the run stopped after the failing step
    # the context still answers: the state reads back (the sweeps gave up
    # before writing, so it is the initial one) and the status stays set
    assert pert_rel_linf(s.q(0), c.q0) < 1e-6
    assert s.sync() == fvna.ERR_TIMEOUT
    s.close()
    # a new context with the default limit takes normal steps, matching the oracle
    q, st = run_gpu(c, 5, precision=fvna.FP32_PERT)
    assert st["rc"] == fvna.OK
    qo, _ = run_oracle(c, 5)
    assert pert_rel_linf(q, qo) <= 1e-5


def test_positive_wait_limit_runs_normally():
    """A generous explicit limit behaves as the default."""
    c = _case()
    q1, st1 = run_gpu(c, 4, precision=fvna.FP32_PERT, wait_limit=1 << 20)
    q2, st2 = run_gpu(c, 4, precision=fvna.FP32_PERT)
    assert st1["rc"] == fvna.OK and st2["rc"] == fvna.OK
    assert np.array_equal(q1, q2)
