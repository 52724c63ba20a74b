"""The per-step boundary-flux budget (fvna_set_budgets, FVNA_FIELD_OUTFLOW):
summed over the cells, the update of eq. fv-hr telescopes to the numerical
fluxes through the border faces, so with extrapolation and periodic borders
(where the source's Laplacian sums to zero) the change of the state's sum
equals minus the accumulated outflow, field by field, up to rounding."""
import numpy as np
import pytest

from paper_1311_3004_gb300 import fvna
from paper_1311_3004_gb300 import workloads as wl

from helpers import Case, gpu_config, gpu_domain

pytestmark = pytest.mark.gpu

P, E, R = fvna.BC_PERIODIC, fvna.BC_EXTRAP, fvna.BC_REFLECT


def _budget_run(prec, bc, steps, q0, nx, ny, splitting=0, tile_x=0):
    c = Case(nx, ny, q0, bc=bc, beta=3.5, delta=2e-3, dx=1.0 / 24)
    s = fvna.Solver(gpu_config(c, prec, splitting=splitting, tile_x=tile_x), [gpu_domain(c)],
                    [q0])
    # binary64 sums the state inside its sweeps (nothing before the first
    # step): the initial sums come from q0; binary32 sums its stored state
    b0 = (np.array([np.sum(q0[0] - 1.0), np.sum(q0[1]), np.sum(q0[2])]) if prec == fvna.FP64
          else s.budget(0))
    s.set_budgets(True)
    s.run(max_steps=steps)
    b1, out = s.budget(0), s.outflow(0)
    s.close()
    return b0, b1, out


@pytest.mark.parametrize("prec", [fvna.FP64, fvna.FP32_PERT])
@pytest.mark.parametrize("splitting", [0, 1])
def test_outflow_balances_the_state_sum_with_extrapolation_borders(prec, splitting):
    """A pulse that reaches every border: the sum of each field changes by
    minus the accumulated outflow (binary64 to 1e-12 of the largest change,
    binary32 to the rounding of its stored perturbations)."""
    n, m = 120, 90
    q0 = wl.gaussian_pulse(n, m, 2e-3, 6.0, seed=3)
    q0 = q0.copy()
    q0[1] += 0.3 * (q0[0] - 1.0)        # a net flow, so that momentum leaves too
    b0, b1, out = _budget_run(prec, (E, E, E, E), 400, q0, n, m, splitting)
    change = b1 - b0
    scale = np.max(np.abs(change))
    assert scale > 1e-4                 # the pulse has left through the borders
    tol = 1e-11 if prec == fvna.FP64 else 2e-5
    assert np.max(np.abs(change + out)) <= tol * scale, (change, -out)


def test_outflow_is_zero_with_periodic_borders():
    n = 64
    q0 = wl.random_smooth(n, n, 2e-3, seed=4)
    b0, b1, out = _budget_run(fvna.FP64, (P, P, P, P), 200, q0, n, n)
    assert np.max(np.abs(out)) <= 1e-14
    assert np.max(np.abs(b1 - b0)) <= 1e-11


def test_outflow_with_the_lanes_along_x1_sweep():
    n, m = 100, 70
    q0 = wl.gaussian_pulse(n, m, 2e-3, 5.0, seed=5)
    b0, b1, out = _budget_run(fvna.FP32_PERT, (E, E, P, P), 300, q0, n, m, tile_x=60)
    change = b1 - b0
    scale = np.max(np.abs(change))
    assert scale > 1e-4
    assert np.max(np.abs(change + out)) <= 2e-5 * scale, (change, -out)
