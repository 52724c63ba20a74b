"""The focused packet of section 4.2 in its two stages on the GPU, through
the C ABI, against the CPU oracle: the driven x1-low border (eq. hifuBC,
packet envelope) feeds the packet in while the domain is at rest; then that
border becomes a zero-order extrapolation (fvna_set_bc) and the window follows
the packet along x1 in whole cells (fvna_shift).  The drive's sin/exp come
from different math libraries on the two sides, so the binary64 bar is a few
ulp of the total state."""
import math

import numpy as np
import pytest

import oracle
from paper_1311_3004_gb300 import analysis, fvna
from paper_1311_3004_gb300 import workloads as wl

from helpers import pert_rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_3004_gb300 import build
    build.build()


def _small():
    # a scaled-down version: F = 10, a = 4, 5 cells per wavelength, 12 x 8 window
    return wl.hifu_cartesian(5.0, 4.0, window=(12.0, 8.0), focal=10.0)


def _oracle_two_stage(w, t_end):
    e = w.extra
    p = oracle.Params(nx=w.nx, ny=w.ny, bc=w.bc, beta=w.beta, delta=w.delta, dx=w.dx,
                      nu_w=w.nu_w, t0=e["t0"], amp=e["amp"], focal=e["focal"],
                      aperture=e["aperture"], envelope=e["envelope"])
    o = oracle.Oracle(p, w.q0)
    switched, moved = False, 0
    while o.scalars()["t"] < t_end:
        o.run(1, t_end)
        t = o.scalars()["t"]
        if not switched and t >= e["t1"]:
            o.set_bc(0, oracle.BC_EXTRAP)
            switched = True
        if switched:
            target = math.floor(1.0 * (t - e["t1"]) / w.dx + 0.5)
            if target > moved:
                o.shift(target - moved, 0)
                moved = target
    q, c, s = o.q(), o.corner(), o.scalars()
    o.close()
    return q, c, s


def _gpu_two_stage(w, t_end, precision):
    e = w.extra
    cfg = fvna.make_config(precision=precision, beta=w.beta, delta=w.delta, dx=w.dx,
                           nu_w=w.nu_w, steps_per_graph=1)
    dom = fvna.make_domain(w.nx, w.ny, bc=w.bc, envelope=e["envelope"], t0=e["t0"], amp=e["amp"],
                           focal=e["focal"], aperture=e["aperture"])
    s = fvna.Solver(cfg, [dom], [w.q0])
    lab_cells = int((t_end - e["t1"] + w.nx * w.dx + 2) / w.dx)
    lab, times, probe = analysis.focused_axis_run(s, w.dx, e["t1"], t_end, e["focal"], lab_cells,
                                                  from_bc=fvna.BC_EXTRAP)
    q, c, st = s.q(0), s.corner(0), s.stats(0)
    s.close()
    return q, c, st, lab


@pytest.mark.parametrize("precision", [fvna.FP64, fvna.FP32_PERT])
def test_two_stage_focused_run_matches_oracle(precision):
    w = _small()
    t_end = 16.0
    qo, co, so = _oracle_two_stage(w, t_end)
    qg, cg, sg, lab = _gpu_two_stage(w, t_end, precision)
    assert so["t"] == t_end and abs(sg["t"] - t_end) < 1e-12
    assert cg[0] > 9.0 and cg == co
    amb = np.zeros_like(qo)
    amb[0] = 1.0
    assert np.max(np.abs(qo - amb)) > 1e-5   # the packet is in the window
    if precision == fvna.FP64:
        assert sg["steps"] == so["step"]
        assert pert_rel_linf(qg, qo) <= 5e-11
        assert np.max(np.abs(qg - qo)) <= 1e-14
    else:
        assert pert_rel_linf(qg, qo) <= 1e-5
    # the on-axis maxima cover the lab cells the window swept, and saw the
    # packet (amplitude of the drive, less the coarse grid's damping)
    swept = int(round(cg[0] / w.dx)) + w.nx
    assert np.all(np.isfinite(lab[:swept])) and np.all(np.isinf(lab[swept:]))
    assert 0.5 * w.extra["amp"] < np.max(lab) < 3.0 * w.extra["amp"]


def test_set_bc_rejects_bad_arguments():
    w = _small()
    e = w.extra
    cfg = fvna.make_config(precision=fvna.FP32_PERT, beta=w.beta, delta=w.delta, dx=w.dx)
    dom = fvna.make_domain(w.nx, w.ny, bc=(fvna.BC_EXTRAP,) * 4)
    s = fvna.Solver(cfg, [dom], [w.q0])
    L = fvna.lib()
    assert L.fvna_set_bc(s._h, 0, 4, fvna.BC_EXTRAP) == fvna.ERR_ARG
    assert L.fvna_set_bc(s._h, 0, 0, 9) == fvna.ERR_ARG
    assert L.fvna_set_bc(s._h, 0, 0, fvna.BC_PERIODIC) == fvna.ERR_ARG   # partner not periodic
    assert L.fvna_set_bc(s._h, 0, 0, fvna.BC_HIFU) == fvna.ERR_ARG       # no ghost ring
    assert L.fvna_set_bc(s._h, 0, 2, fvna.BC_REFLECT) == fvna.OK
    s.close()
