"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds initial states and parameter sets.  It holds none of
the scheme's arithmetic, so that the GPU path and the CPU oracle can both be
fed from it.  States are numpy arrays of shape (3, ny, nx) in the paper's
dimensionless total variables q = (rho/rho0)(1, u1/c0, u2/c0) (eq. adim:q).

Physical units are converted once here (eqs. renorm and phi-tdelta):
    beta = 1 + B/(2A),   dt~ = delta / (c0 L),   A = p_amp / (rho0 c0^2),
with L the wavelength c0/f for the plane-wave and focused-source cases.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Water (the plane-wave configuration names it; assumed for the others).
RHO0 = 1000.0        # kg/m^3
C0 = 1500.0          # m/s
B_OVER_A = 5.0
DIFFUSIVITY = 4.3e-6  # m^2/s, sound diffusivity delta


def beta_of(b_over_a: float = B_OVER_A) -> float:
    return 1.0 + 0.5 * b_over_a


def delta_tilde(freq_hz: float, diffusivity: float = DIFFUSIVITY, c0: float = C0) -> float:
    """dt~ = delta/(c0 L) with L = c0/f (one wavelength)."""
    return diffusivity / (c0 * (c0 / freq_hz))


def amplitude(p_pa: float, rho0: float = RHO0, c0: float = C0) -> float:
    """Dimensionless density perturbation of a pressure amplitude, p = c0^2 rho."""
    return p_pa / (rho0 * c0 * c0)


def ambient(nx: int, ny: int) -> np.ndarray:
    q = np.zeros((3, ny, nx), dtype=np.float64)
    q[0] = 1.0
    return q


def cell_centres(nx: int, ny: int, dx: float, x0: float = 0.0, y0: float = 0.0):
    x = x0 + (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dx
    return np.meshgrid(x, y)  # each (ny, nx)


def plane_sine(nx: int, ny: int, amp: float, cells_per_wavelength: float) -> np.ndarray:
    """Right-going sinusoid along x1: q1 = 1 + A sin(2 pi x), q2 = q1 - 1, q3 = 0
    (the small-signal right-going relation of eq. OurTaylorS)."""
    X, _ = cell_centres(nx, ny, 1.0 / cells_per_wavelength)
    q = ambient(nx, ny)
    q[0] = 1.0 + amp * np.sin(2.0 * np.pi * X)
    q[1] = q[0] - 1.0
    return q


def gaussian_pulse(nx: int, ny: int, amp: float, sigma_cells: float, seed: int,
                   max_offset_cells: int = 256) -> np.ndarray:
    """Pressure Gaussian exp(-r^2/(2 sigma^2)) at rest, centre offset drawn from seed."""
    rng = np.random.default_rng(seed)
    off = min(max_offset_cells, max(0, min(nx, ny) // 2 - 4 * int(sigma_cells) - 1))
    cx = nx / 2.0 + rng.integers(-off, off + 1)
    cy = ny / 2.0 + rng.integers(-off, off + 1)
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    I, J = np.meshgrid(i, j)
    r2 = (I - cx) ** 2 + (J - cy) ** 2
    q = ambient(nx, ny)
    q[0] = 1.0 + amp * np.exp(-r2 / (2.0 * sigma_cells ** 2))
    return q


def centred_gaussian(nx: int, ny: int, amp: float, sigma_cells: float) -> np.ndarray:
    """Gaussian exactly at the domain centre (for mirror-symmetry checks)."""
    i = np.arange(nx) + 0.5 - nx / 2.0
    j = np.arange(ny) + 0.5 - ny / 2.0
    I, J = np.meshgrid(i, j)
    q = ambient(nx, ny)
    q[0] = 1.0 + amp * np.exp(-(I * I + J * J) / (2.0 * sigma_cells ** 2))
    return q


def random_smooth(nx: int, ny: int, amp: float, seed: int, modes: int = 4) -> np.ndarray:
    """Sum of a few random Fourier modes in all three fields (periodic-friendly)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)
    q = ambient(nx, ny)
    for k in range(3):
        f = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(0, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
        q[k] += amp * f / modes
    return q


def random_cells(nx: int, ny: int, amp: float, seed: int) -> np.ndarray:
    """Independent uniform perturbations per cell (rough data; exercises the limiter)."""
    rng = np.random.default_rng(seed)
    q = ambient(nx, ny)
    q += amp * rng.uniform(-1.0, 1.0, size=q.shape)
    return q


def taylor_initial(nx: int, ny: int, dx: float, ratio: float, x0: float = 0.0,
                   y0: float = 0.0, angle: float = 0.0, t: float = 0.0) -> np.ndarray:
    """Taylor-shock profile of eq. OurTaylorS at time t (rotated by angle)."""
    X, Y = cell_centres(nx, ny, dx, x0, y0)
    c, s = np.cos(angle), np.sin(angle)
    q = ambient(nx, ny)
    q[0] = 1.0 - ratio * np.tanh(X * c + Y * s - t)
    q[1] = (q[0] - 1.0) * c
    q[2] = (q[0] - 1.0) * s
    return q


def tone_burst(nx: int, ny: int, amp: float, cells_per_wavelength: float, angle: float,
               cycles: float = 4.0, centre=None) -> np.ndarray:
    """Gaussian-enveloped plane tone burst travelling at `angle` (small-signal relation)."""
    dx = 1.0 / cells_per_wavelength
    X, Y = cell_centres(nx, ny, dx)
    if centre is None:
        centre = (nx * dx / 2.0, ny * dx / 2.0)
    c, s = np.cos(angle), np.sin(angle)
    xi = (X - centre[0]) * c + (Y - centre[1]) * s
    w = amp * np.sin(2 * np.pi * xi) * np.exp(-(xi / (cycles / 2.0)) ** 2)
    q = ambient(nx, ny)
    q[0] = 1.0 + w
    q[1] = w * c
    q[2] = w * s
    return q


@dataclass
class Workload:
    """A named configuration: sizes, parameters and a state generator."""
    name: str
    nx: int
    ny: int
    steps: int
    beta: float
    delta: float
    dx: float
    nu_w: float
    bc: tuple
    q0: np.ndarray
    geometry: int = 0
    extra: dict = None


BC_PERIODIC, BC_EXTRAP, BC_REFLECT, BC_TAYLOR, BC_HIFU = 0, 1, 2, 3, 4


def plane_wave_512x8(steps: int = 2000) -> Workload:
    """Plane-wave shock formation: 512x8 cells, periodic in y, extrapolation in
    x, water, 1 MHz, 1 MPa, 40 cells per wavelength, MC limiter, CFL 0.9."""
    eta = 40
    q0 = plane_sine(512, 8, amplitude(1.0e6), eta)
    return Workload("plane_wave_512x8", 512, 8, steps, beta_of(), delta_tilde(1.0e6),
                    1.0 / eta, 0.9, (BC_EXTRAP, BC_EXTRAP, BC_PERIODIC, BC_PERIODIC), q0)


def gaussian_2048(steps: int = 5000, n: int = 2048, seed: int = 2) -> Workload:
    """2D Cartesian Gaussian pulse: n x n cells (2048^2 by default), peak 2 MPa,
    sigma 8 cells, centre offset from the seed, extrapolation borders, 40 cells
    per wavelength at 1 MHz (dx = 37.5 um)."""
    eta = 40
    q0 = gaussian_pulse(n, n, amplitude(2.0e6), 8.0, seed)
    return Workload(f"gaussian_{n}x{n}", n, n, steps, beta_of(), delta_tilde(1.0e6),
                    1.0 / eta, 0.9, (BC_EXTRAP,) * 4, q0)


def focused_axisym(nz: int = 4096, nr: int = 1024, cells_per_wavelength: float = 30.0,
                   p_surface: float = 0.3e6, freq: float = 1.0e6, aperture_m: float = 30e-3,
                   focal_m: float = 60e-3, transits: float = 8.0) -> Workload:
    """Axisymmetric focused-source field in (z, r): a curved aperture of radius
    30 mm and focal length 60 mm driven sinusoidally at 1 MHz on the z = 0
    border (reflective axis at r = 0, extrapolation elsewhere), water, 30 cells
    per wavelength, run for `transits` focal transit times (quasi-steady).
    L = one wavelength, so the aperture is 20 and the focal length 40."""
    lam = C0 / freq
    q0 = ambient(nz, nr)
    # CFL 0.4: with the first-order flux on the two radial faces next to the
    # axis, the linearised axisymmetric step is stable up to CFL 0.5
    w = Workload(f"focused_axisym_{nz}x{nr}", nz, nr, 0, beta_of(), delta_tilde(freq),
                 1.0 / cells_per_wavelength, 0.4, (BC_HIFU, BC_EXTRAP, BC_REFLECT, BC_EXTRAP), q0,
                 geometry=1,
                 extra={"amp": amplitude(p_surface), "focal": focal_m / lam,
                        "aperture": aperture_m / lam, "envelope": 0,
                        "t_end": transits * focal_m / lam})
    return w


def batched_64(seed: int = 4, n_domains: int = 64, n_min: int = 256, n_max: int = 1536):
    """Many independent domains of uneven size: square sides uniform in
    [n_min, n_max], amplitudes log-uniform in [0.1, 2] MPa, frequencies uniform
    in [0.5, 2] MHz, each a 4-cycle Gaussian tone burst at a seeded angle,
    extrapolation borders, one common cell size of 37.5 um (L = 1.5 mm, the
    1 MHz wavelength, so dx = 1/40 and the burst wavelength is 1/f[MHz]).
    Returns (list of (nx, ny, q0, info), beta, delta, dx)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / 40.0
    out = []
    for k in range(n_domains):
        n = int(rng.integers(n_min, n_max + 1))
        p = float(np.exp(rng.uniform(np.log(0.1e6), np.log(2.0e6))))
        f = float(rng.uniform(0.5e6, 2.0e6))
        ang = float(rng.uniform(0.0, 2.0 * np.pi))
        q0 = tone_burst(n, n, amplitude(p), (1.0e6 / f) / dx, ang)
        out.append((n, n, q0, {"p_pa": p, "f_hz": f, "angle": ang}))
    return out, beta_of(), delta_tilde(1.0e6), dx


# Soft tissue, section 4.2 (after Albin et al.): delta = 6.4117e-4 m^2/s,
# c0 = 1540 m/s, f0 = 1.1 MHz, beta = 4.8; L = one wavelength.
def hifu_cartesian(eta: float, aperture: float, window=None, focal: float = 50.0,
                   amp: float = 4.217e-4, delta: float = 2.974e-4, beta: float = 4.8) -> Workload:
    """The focused packet of section 4.2 in the 2D Cartesian half plane x2 >= 0:
    a circular-arc transducer of focal length F and half aperture a drives the
    x1 = 0 border for 0 <= x2 <= a with the packet of eq. hifuBC (envelope
    exp(-(tau/4)^10)), the x2 = 0 border is a symmetry (reflective) axis, the
    other borders extrapolate.  `window` = (length along x1, height) in
    wavelengths (default (28, a + 10)).  The run starts at t0, when the packet
    is zero to binary64 precision at every driven point: exp(-(tau/4)^10) <
    1e-16 for |tau| > 5.74, and tau = t + x2^2/(2F) reaches -5.74 first at
    x2 = a.  extra["t1"] is the end of the first stage: the packet has fully
    entered on the axis (tau > 5.74 at x1 = 0, x2 = 0)."""
    lx, ly = window if window is not None else (28.0, aperture + 10.0)
    nx, ny = int(round(lx * eta)), int(round(ly * eta))
    t0 = -(5.74 + aperture * aperture / (2.0 * focal)) - 0.5
    return Workload(f"hifu_cartesian_a{aperture:g}_eta{eta:g}", nx, ny, 0, beta, delta, 1.0 / eta,
                    0.9, (BC_HIFU, BC_EXTRAP, BC_REFLECT, BC_EXTRAP), ambient(nx, ny),
                    extra={"amp": amp, "focal": focal, "aperture": aperture, "envelope": 1,
                           "t0": t0, "t1": 6.0})


# ---------------------------------------------------------------- three dimensions

def ambient3(nx: int, ny: int, nz: int) -> np.ndarray:
    """State at rest in 3D: (4, nz, ny, nx) with q1 = 1."""
    q = np.zeros((4, nz, ny, nx))
    q[0] = 1.0
    return q


def gaussian_pulse3(nx: int, ny: int, nz: int, amp: float, sigma_cells: float, seed: int,
                    max_offset: float = 0.125) -> np.ndarray:
    """3D Gaussian pressure pulse at rest: q1 = 1 + amp exp(-r^2 / (2 sigma^2)),
    the centre offset from the box centre by a seeded fraction (up to
    max_offset of each side)."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(-max_offset, max_offset, size=3)
    c = [(n / 2.0) * (1.0 + 2.0 * o) for n, o in zip((nx, ny, nz), off)]
    z = (np.arange(nz) + 0.5 - c[2])[:, None, None]
    y = (np.arange(ny) + 0.5 - c[1])[None, :, None]
    x = (np.arange(nx) + 0.5 - c[0])[None, None, :]
    q = ambient3(nx, ny, nz)
    q[0] += amp * np.exp(-(x * x + y * y + z * z) / (2.0 * sigma_cells ** 2))
    return q


def random_smooth3(nx: int, ny: int, nz: int, amp: float, seed: int, modes: int = 4) -> np.ndarray:
    """Sum of a few random Fourier modes in all four fields (periodic-friendly)."""
    rng = np.random.default_rng(seed)
    z = (np.arange(nz) / nz)[:, None, None]
    y = (np.arange(ny) / ny)[None, :, None]
    x = (np.arange(nx) / nx)[None, None, :]
    q = ambient3(nx, ny, nz)
    for f in range(4):
        acc = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            acc += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * x + ky * y + kz * z) + ph)
        q[f] += amp * acc / modes
    return q


def gaussian3d(n: int = 256, seed: int = 2) -> dict:
    """The 2D pulse workload's 3D counterpart: an n^3 box (256^3 by default),
    peak 2 MPa, sigma 8 cells, centre offset from the seed, extrapolation on
    all six faces, water at 1 MHz with 40 cells per wavelength."""
    return {"name": f"gaussian3d_{n}", "n": n, "q0": gaussian_pulse3(n, n, n, amplitude(2.0e6), 8.0,
                                                                      seed),
            "beta": beta_of(), "delta": delta_tilde(1.0e6), "dx": 1.0 / 40, "nu_w": 0.9,
            "bc": (BC_EXTRAP,) * 6}
