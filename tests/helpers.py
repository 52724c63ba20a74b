"""Shared helpers of the GPU tests: one description of a run, executed both by
the CPU oracle and by the CUDA library through the C ABI, and the error
measures the comparisons use."""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

import oracle
from paper_1311_3004_gb300 import fvna


@dataclass
class Case:
    nx: int
    ny: int
    q0: np.ndarray
    bc: tuple = (1, 1, 1, 1)
    beta: float = 3.5
    delta: float = 0.0
    dx: float = 1.0 / 32
    nu_w: float = 0.9
    nu_max: float = 1.0
    dt_fixed: float = 0.0
    limiter: int = 0
    sweeps: int = 7
    geometry: int = 0
    envelope: int = 0
    x0: float = 0.0
    y0: float = 0.0
    t0: float = 0.0
    taylor_ratio: float = 0.0
    taylor_angle: float = 0.0
    amp: float = 0.0
    focal: float = 1.0
    aperture: float = 0.0


def oracle_params(c: Case) -> oracle.Params:
    return oracle.Params(nx=c.nx, ny=c.ny, bc=tuple(c.bc), limiter=c.limiter, sweeps=c.sweeps,
                         geometry=c.geometry, envelope=c.envelope, beta=c.beta, delta=c.delta,
                         dx=c.dx, nu_w=c.nu_w, nu_max=c.nu_max, dt_fixed=c.dt_fixed, x0=c.x0,
                         y0=c.y0, t0=c.t0, taylor_ratio=c.taylor_ratio,
                         taylor_angle=c.taylor_angle, amp=c.amp, focal=c.focal,
                         aperture=c.aperture)


def gpu_config(c: Case, precision=fvna.FP64, **kw) -> fvna.Config:
    return fvna.make_config(precision=precision, geometry=c.geometry, limiter=c.limiter,
                            sweeps=c.sweeps, beta=c.beta, delta=c.delta, dx=c.dx, nu_w=c.nu_w,
                            nu_max=c.nu_max, dt_fixed=c.dt_fixed, **kw)


def gpu_domain(c: Case, dt0: float = 0.0, t0: float = None) -> fvna.Domain:
    return fvna.make_domain(c.nx, c.ny, bc=c.bc, envelope=c.envelope, x0=c.x0, y0=c.y0,
                            t0=c.t0 if t0 is None else t0, dt0=dt0,
                            taylor_ratio=c.taylor_ratio, taylor_angle=c.taylor_angle, amp=c.amp,
                            focal=c.focal, aperture=c.aperture)


def run_oracle(c: Case, steps: int, t_end: float = -np.inf):
    return oracle.run(oracle_params(c), c.q0, steps, t_end)


def run_gpu(c: Case, steps: int, t_end: float = -np.inf, precision=fvna.FP64, **kw):
    s = fvna.Solver(gpu_config(c, precision, **kw), [gpu_domain(c)], [c.q0])
    st = s.run(t_end=t_end, max_steps=steps, check=False)
    q = s.q(0)
    s.close()
    return q, st


def pert_rel_linf(q, ref, q_amb=None):
    """max over fields |q - ref| / max over fields |ref - ambient| (perturbation-relative)."""
    amb = np.zeros_like(ref)
    amb[0] = 1.0
    scale = np.max(np.abs(ref - amb))
    return float(np.max(np.abs(q - ref)) / scale) if scale > 0 else float(np.max(np.abs(q - ref)))


def pressure_errors(p, pref):
    """Relative peak-pressure error and relative L2 error of p against pref."""
    peak = abs(np.max(np.abs(p)) - np.max(np.abs(pref))) / np.max(np.abs(pref))
    l2 = np.linalg.norm(p - pref) / np.linalg.norm(pref)
    return float(peak), float(l2)
