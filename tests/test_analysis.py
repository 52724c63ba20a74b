"""Host-side evaluation helpers (section 4.1 error line, section 4.2 spectrum)
against values they must reproduce exactly or to quadrature accuracy."""
import math

import numpy as np
import pytest

from paper_1311_3004_gb300 import analysis
from paper_1311_3004_gb300 import workloads as wl


@pytest.mark.parametrize("angle", [0.0, math.pi / 32, math.pi / 8, math.pi / 4])
def test_line_errors_vanish_on_the_analytic_profile(angle):
    eta, ratio, t = 20, 1e-7, 3.0
    dx, n = 1.0 / eta, 240
    x0 = y0 = -6.0
    q = wl.taylor_initial(n, n, dx, ratio, x0=x0 + t * math.cos(angle),
                          y0=y0 + t * math.sin(angle), angle=angle, t=t)
    e1, einf = analysis.taylor_line_errors(q, x0 + t * math.cos(angle), y0 + t * math.sin(angle),
                                           dx, t, angle, ratio)
    # exact at cell centres (theta = 0) up to the rounding of q1 = 1 + O(1e-7)
    # (1e-16 / 1e-7 relative); bilinear sampling of tanh otherwise
    bound = 1e-8 if angle == 0.0 else 0.25 * dx * dx
    assert e1 <= bound and einf <= 4 * bound


def test_line_errors_measure_a_shift():
    """A profile displaced by d along the propagation direction has E_1 equal
    to the L1 distance of the two tanh curves over the line, relative."""
    eta, ratio, t, d = 40, 1e-7, 0.0, 0.05
    dx, n = 1.0 / eta, 480
    q = wl.taylor_initial(n, 4, dx, ratio, x0=-6.0, t=t + d)
    e1, _ = analysis.taylor_line_errors(q, -6.0, 0.0, dx, t, 0.0, ratio)
    x = -6.0 + (np.arange(n) + 0.5) * dx
    sel = np.abs(x - t) <= 5.0
    ref = np.sum(np.abs(np.tanh(x[sel] - t - d) - np.tanh(x[sel] - t))) / np.sum(
        np.abs(np.tanh(x[sel] - t)))
    assert e1 == pytest.approx(ref, rel=1e-7)   # q1 - 1 carries 1e-16 / 1e-7 rounding


def test_convergence_rate_of_a_power_law():
    etas = [5, 10, 20, 41, 82]
    assert analysis.convergence_rate(etas, [3.0 * e ** -1.7 for e in etas]) == pytest.approx(1.7)


def test_harmonics_of_a_distorted_sine():
    """Uneven sampling of 0.4 sin(2 pi t) + 0.1 sin(4 pi t + 0.3) over 40 periods."""
    rng = np.random.default_rng(0)
    t = np.cumsum(rng.uniform(0.009, 0.011, 4000))
    v = 0.4 * np.sin(2 * np.pi * t) + 0.1 * np.sin(4 * np.pi * t + 0.3)
    h = analysis.harmonics(t, v, 4)
    assert h[0] == pytest.approx(0.4, rel=0.02)
    assert h[1] == pytest.approx(0.1, rel=0.05)
    assert h[2] < 0.01 and h[3] < 0.01


def test_bias_slices_cover_the_biases_of_the_flat_layout():
    """The bias-free training option zeroes exactly b1, b2 and b3 of the
    flat parameter layout (w1 b1 w2 b2 w3 b3) and nothing else."""
    from paper_1311_3004_gb300 import fvna, learned
    flat = np.arange(fvna.NET_PARAMS, dtype=np.float32) + 1.0
    for sl in learned._bias_slices():
        flat[sl] = 0.0
    d = fvna.net_params_dict(flat)
    for k in ("b1", "b2", "b3"):
        assert np.all(d[k] == 0.0), k
    for k in ("w1", "w2", "w3"):
        assert np.all(d[k] != 0.0), k
