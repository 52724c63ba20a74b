"""Post-processing of solver output: the error measures of section 4.1.

The Taylor-shock errors of eq. error compare the numerical q1 - 1 with the
analytic profile of eq. OurTaylorS, -(dt~/beta) tanh(x . n - t), on a 10-unit
line along the propagation direction n = (cos theta_T, sin theta_T), centred on
the shock: E_1 = |num - ref|_1 / |ref|_1 and E_inf = |num - ref|_inf /
|ref|_inf.  The line is sampled at cell centres when it runs along a grid row
(theta_T = 0) and bilinearly otherwise.  This is host-side evaluation of a
result (numpy), not part of the scheme.
"""
from __future__ import annotations

import math

import numpy as np


def taylor_line_errors(q: np.ndarray, x0: float, y0: float, dx: float, t: float, angle: float,
                       ratio: float, half: float = 5.0, samples: int = 401):
    """(E_1, E_inf) of the state q (3, ny, nx; total variables) of a window with
    lower-left corner (x0, y0), at time t.  The line passes through the point of
    the shock (x . n = t) nearest to the window centre."""
    ny, nx = q.shape[1:]
    ct, st = math.cos(angle), math.sin(angle)
    f = q[0] - 1.0
    if angle == 0.0:
        x = x0 + (np.arange(nx) + 0.5) * dx
        row = ny // 2
        sel = np.abs(x - t) <= half
        num = f[row, sel]
        ref = -ratio * np.tanh(x[sel] - t)
    else:
        cx, cy = x0 + 0.5 * nx * dx, y0 + 0.5 * ny * dx
        s0 = cx * ct + cy * st
        cx, cy = cx + (t - s0) * ct, cy + (t - s0) * st
        s = np.linspace(-half, half, samples)
        px, py = cx + s * ct, cy + s * st
        fi, fj = (px - x0) / dx - 0.5, (py - y0) / dx - 0.5
        i0, j0 = np.floor(fi).astype(int), np.floor(fj).astype(int)
        if i0.min() < 0 or j0.min() < 0 or i0.max() + 1 >= nx or j0.max() + 1 >= ny:
            raise ValueError("the error line leaves the window")
        a, b = fi - i0, fj - j0
        num = ((1 - a) * (1 - b) * f[j0, i0] + a * (1 - b) * f[j0, i0 + 1]
               + (1 - a) * b * f[j0 + 1, i0] + a * b * f[j0 + 1, i0 + 1])
        ref = -ratio * np.tanh(s)
    e1 = float(np.sum(np.abs(num - ref)) / np.sum(np.abs(ref)))
    einf = float(np.max(np.abs(num - ref)) / np.max(np.abs(ref)))
    return e1, einf


def convergence_rate(etas, errors) -> float:
    """Slope of the linear regression of log(E) on log(eta), negated (section 4.1)."""
    return float(-np.polyfit(np.log(np.asarray(etas, float)), np.log(np.asarray(errors, float)),
                             1)[0])


def focused_axis_run(solver, dx: float, t1: float, t_end: float, probe_x1: float,
                     lab_cells: int, extrapolate_side: int = 0, from_bc: int = 1,
                     velocity: float = 1.0, central: bool = False):
    """The two stages of section 4.2 on a fvna.Solver holding one domain whose
    x2-low border is the symmetry axis: step by step until t1 with the domain
    at rest; then the driven x1-low border becomes a zero-order extrapolation
    (rule `from_bc`) and the window follows the packet at `velocity` along
    x1 in whole cells.  After every step the pressure along the axis (row 0)
    updates the running maximum of each lab-frame cell (the on-axis pressure
    maxima of the section) and the pressure at the lab point (probe_x1, 0) is
    recorded.  Returns (axis maxima over lab cells 0..lab_cells-1, times,
    probe pressures); with central=True also the maxima of the packet's
    central peak (section 4.2 measures the maximum pressure on the central
    peak of the packet, away from its transitory head and tail): at each lab
    cell the maximum over the one period centred on the passage of the
    packet's centre, which on the axis reaches x1 at t = x1 (tau = t - x1 in
    eq. hifuBC), i.e. over |t - x1| <= 1/2."""
    lab = np.full(lab_cells, -np.inf)
    cen = np.full(lab_cells, -np.inf)
    times, probe = [], []
    switched, moved = False, 0
    t = solver.stats(0)["t"]
    while t < t_end:
        st = solver.run(t_end=t_end, max_steps=1)
        t = st["t"]
        if not switched and t >= t1:
            solver.set_bc(0, extrapolate_side, from_bc)
            switched = True
        if switched:
            target = int(math.floor(velocity * (t - t1) / dx + 0.5))
            if target > moved:
                solver.shift(0, target - moved, 0)
                moved = target
        p = solver.axis_pressure(0)
        k0 = moved
        n = min(len(p), lab_cells - k0)
        if n > 0:
            np.maximum(lab[k0:k0 + n], p[:n], out=lab[k0:k0 + n])
            if central:
                x = (np.arange(k0, k0 + n) + 0.5) * dx
                inside = np.abs(t - x) <= 0.5
                cen[k0:k0 + n] = np.where(inside, np.maximum(cen[k0:k0 + n], p[:n]),
                                          cen[k0:k0 + n])
        ip = int(math.floor(probe_x1 / dx)) - k0
        if 0 <= ip < len(p):
            times.append(t)
            probe.append(p[ip])
    if central:
        return lab, np.asarray(times), np.asarray(probe), cen
    return lab, np.asarray(times), np.asarray(probe)


def harmonics(times, values, n: int = 8):
    """Amplitudes of harmonics 1..n (fundamental frequency 1) of a signal sampled
    at uneven times: linear resampling onto a uniform grid of the mean spacing,
    then an FFT; amplitudes at the bins nearest the integer frequencies."""
    times = np.asarray(times, float)
    values = np.asarray(values, float)
    dt = float(np.mean(np.diff(times)))
    tu = np.arange(times[0], times[-1], dt)
    vu = np.interp(tu, times, values)
    spec = np.abs(np.fft.rfft(vu)) * 2.0 / len(vu)
    freq = np.fft.rfftfreq(len(vu), dt)
    return [float(spec[int(np.argmin(np.abs(freq - k)))]) for k in range(1, n + 1)]
