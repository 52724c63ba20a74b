"""Plain FP64 CPU oracle of the arXiv 1311.3004 finite-volume scheme.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports or calls anything here, and this package imports nothing from it.

The arithmetic lives in ``fvna_oracle.c`` (the paper's 2D scheme) and
``fvna_oracle3d.c`` (its three-dimensional form), plain C, binary64,
``-ffp-contract=off``; this module compiles them with gcc and wraps them with
ctypes.  See the headers of the C files for what each function follows in
the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fvna_oracle.c")
_SRC3 = os.path.join(_HERE, "fvna_oracle3d.c")
_LIB = os.path.join(_HERE, "_build", "libfvna_oracle.so")

BC_PERIODIC, BC_EXTRAP, BC_REFLECT, BC_TAYLOR, BC_HIFU = 0, 1, 2, 3, 4
LIM_MC, LIM_NONE, LIM_LW = 0, 1, 2
ST_NONREAL, ST_CFL, ST_NAN = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    srcs = [_SRC, _SRC3]
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in srcs):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("limiter", ctypes.c_int), ("sweeps", ctypes.c_int), ("geometry", ctypes.c_int),
                ("envelope", ctypes.c_int),
                ("beta", ctypes.c_double), ("delta", ctypes.c_double), ("dx", ctypes.c_double),
                ("nu_w", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("t0", ctypes.c_double), ("taylor_ratio", ctypes.c_double),
                ("taylor_angle", ctypes.c_double), ("amp", ctypes.c_double),
                ("focal", ctypes.c_double), ("aperture", ctypes.c_double),
                ("splitting", ctypes.c_int), ("reserved", ctypes.c_int)]


class _Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 6), ("limiter", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("beta", ctypes.c_double), ("delta", ctypes.c_double), ("dx", ctypes.c_double),
                ("nu_w", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("t0", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.ora_create.restype = ctypes.c_void_p
        L.ora_create.argtypes = [ctypes.POINTER(_Params), dp]
        L.ora_destroy.argtypes = [ctypes.c_void_p]
        L.ora_run.restype = ctypes.c_long
        L.ora_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_long]
        L.ora_get.argtypes = [ctypes.c_void_p, dp]
        L.ora_scalars.argtypes = [ctypes.c_void_p, dp]
        L.ora_interface.restype = ctypes.c_int
        L.ora_interface.argtypes = [ctypes.c_double, dp, dp, dp, dp, dp, dp]
        L.ora_shift.restype = ctypes.c_int
        L.ora_shift.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.ora_corner.argtypes = [ctypes.c_void_p, dp]
        L.ora_set_bc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.ora_drive.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, dp]
        L.ora_limiter.restype = ctypes.c_double
        L.ora_limiter.argtypes = [ctypes.c_int, ctypes.c_double]
        L.ora3_create.restype = ctypes.c_void_p
        L.ora3_create.argtypes = [ctypes.POINTER(_Params3), dp]
        L.ora3_destroy.argtypes = [ctypes.c_void_p]
        L.ora3_run.restype = ctypes.c_long
        L.ora3_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_long]
        L.ora3_get.argtypes = [ctypes.c_void_p, dp]
        L.ora3_scalars.argtypes = [ctypes.c_void_p, dp]
        L.ora3_interface.restype = ctypes.c_int
        L.ora3_interface.argtypes = [ctypes.c_double, dp, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """One run's parameters (all dimensionless, see eq. renorm)."""
    nx: int
    ny: int
    bc: tuple = (BC_EXTRAP, BC_EXTRAP, BC_EXTRAP, BC_EXTRAP)
    limiter: int = LIM_MC
    sweeps: int = 7
    geometry: int = 0
    envelope: int = 0
    beta: float = 3.5
    delta: float = 0.0
    dx: float = 1.0
    nu_w: float = 0.9
    nu_max: float = 1.0
    dt_fixed: float = 0.0
    x0: float = 0.0
    y0: float = 0.0
    t0: float = 0.0
    taylor_ratio: float = 0.0
    taylor_angle: float = 0.0
    amp: float = 0.0
    focal: float = 1.0
    aperture: float = 0.0
    splitting: int = 0          # 0 Godunov, 1 Strang
    reserved: int = 0

    def to_c(self) -> _Params:
        p = _Params()
        for f in _Params._fields_:
            name = f[0]
            if name == "bc":
                p.bc = (ctypes.c_int * 4)(*self.bc)
            else:
                setattr(p, name, getattr(self, name))
        return p


class Oracle:
    """A running oracle state.  q0 has shape (3, ny, nx), total variables."""

    def __init__(self, params: Params, q0: np.ndarray):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        assert q0.shape == (3, params.ny, params.nx)
        self.params = params
        self._p = params.to_c()
        self._h = lib().ora_create(ctypes.byref(self._p), _dptr(q0))

    def run(self, steps: int, t_end: float = -np.inf) -> int:
        t_end = float(t_end) if np.isfinite(t_end) else -1e300
        return int(lib().ora_run(self._h, t_end, int(steps)))

    def shift(self, kx: int, ky: int) -> None:
        """Move the window by (kx, ky) cells (moving domain, see ora_shift)."""
        if lib().ora_shift(self._h, int(kx), int(ky)) != 0:
            raise ValueError(f"shift ({kx}, {ky}) out of range")

    def set_bc(self, side: int, bc: int) -> None:
        """Border rule of one side from the next step on."""
        lib().ora_set_bc(self._h, int(side), int(bc))

    def corner(self) -> tuple:
        out = np.zeros(2, dtype=np.float64)
        lib().ora_corner(self._h, _dptr(out))
        return float(out[0]), float(out[1])

    def q(self) -> np.ndarray:
        out = np.empty((3, self.params.ny, self.params.nx), dtype=np.float64)
        lib().ora_get(self._h, _dptr(out))
        return out

    def scalars(self) -> dict:
        out = np.zeros(9, dtype=np.float64)
        lib().ora_scalars(self._h, _dptr(out))
        keys = ["t", "dt", "smax", "nu_min", "nu_max", "nu_mean", "nu_std", "step", "status"]
        d = dict(zip(keys, out.tolist()))
        d["step"] = int(d["step"])
        d["status"] = int(d["status"])
        return d

    def close(self):
        if getattr(self, "_h", None):
            lib().ora_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def interface(beta: float, qL, qR):
    """One x1-sweep interface: (s[3], W[3,3] rows = families, amdq[3], apdq[3], nonreal)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    s = np.zeros(3)
    W = np.zeros(9)
    am = np.zeros(3)
    ap = np.zeros(3)
    nr = lib().ora_interface(beta, _dptr(qL), _dptr(qR), _dptr(s), _dptr(W), _dptr(am), _dptr(ap))
    return s, W.reshape(3, 3), am, ap, bool(nr)


def drive(params: Params, x1: float, x2: float, t: float) -> np.ndarray:
    """Border values (q1, q2, q3) of the focused drive of eq. hifuBC at (x1, x2)
    and time t, with the amplitude, focal length and envelope of `params`."""
    p = params.to_c()
    out = np.zeros(3)
    lib().ora_drive(ctypes.byref(p), float(x1), float(x2), float(t), _dptr(out))
    return out


def limiter(kind: int, theta: float) -> float:
    return float(lib().ora_limiter(kind, theta))


def run_moving(o: Oracle, t_end: float, t1: float, velocity, every: int,
               max_steps: int = 2 ** 62) -> None:
    """Two-stage run with a moving window (section 4: the domain is at rest
    until t1, then moves with the wave).  The run goes in chunks of `every`
    steps; after each chunk the window is moved by whole cells so that its
    displacement since the start is (round(v_x (t - t1) / dx), round(v_y (t -
    t1) / dx)).  Stops at t_end, after max_steps steps, or on a nonzero
    status."""
    dx = o.params.dx
    timed = t_end > o.scalars()["t"]
    moved = [0, 0]
    left = int(max_steps)
    while left > 0:
        n = min(int(every), left)
        o.run(n, t_end)
        left -= n
        sc = o.scalars()
        if sc["status"]:
            break
        if sc["t"] > t1:
            e = sc["t"] - t1
            tx = int(np.floor(velocity[0] * e / dx + 0.5))
            ty = int(np.floor(velocity[1] * e / dx + 0.5))
            if tx != moved[0] or ty != moved[1]:
                o.shift(tx - moved[0], ty - moved[1])
                moved = [tx, ty]
        if timed and not sc["t"] < t_end:
            break


def run(params: Params, q0: np.ndarray, steps: int, t_end: float = -np.inf):
    """Convenience: run and return (q, scalars)."""
    o = Oracle(params, q0)
    o.run(steps, t_end)
    q, sc = o.q(), o.scalars()
    o.close()
    return q, sc


# ---------------------------------------------------------------- three dimensions

@dataclass
class Params3:
    """One 3D run's parameters (fvna_oracle3d.c).  sweeps: bit 0 x1, bit 1 x2,
    bit 2 x3, bit 3 source; bc: x1-low, x1-high, x2-low, x2-high, x3-low,
    x3-high, each periodic, extrapolation or reflective."""
    nx: int
    ny: int
    nz: int
    bc: tuple = (BC_EXTRAP,) * 6
    limiter: int = LIM_MC
    sweeps: int = 15
    beta: float = 3.5
    delta: float = 0.0
    dx: float = 1.0
    nu_w: float = 0.9
    nu_max: float = 1.0
    dt_fixed: float = 0.0
    t0: float = 0.0

    def to_c(self) -> _Params3:
        p = _Params3()
        for name, _ in _Params3._fields_:
            if name == "bc":
                p.bc = (ctypes.c_int * 6)(*self.bc)
            else:
                setattr(p, name, getattr(self, name))
        return p


class Oracle3:
    """A running 3D oracle state.  q0 has shape (4, nz, ny, nx), total variables."""

    def __init__(self, params: Params3, q0: np.ndarray):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        assert q0.shape == (4, params.nz, params.ny, params.nx)
        self.params = params
        self._p = params.to_c()
        self._h = lib().ora3_create(ctypes.byref(self._p), _dptr(q0))

    def run(self, steps: int, t_end: float = -np.inf) -> int:
        t_end = float(t_end) if np.isfinite(t_end) else -1e300
        return int(lib().ora3_run(self._h, t_end, int(steps)))

    def q(self) -> np.ndarray:
        p = self.params
        out = np.empty((4, p.nz, p.ny, p.nx), dtype=np.float64)
        lib().ora3_get(self._h, _dptr(out))
        return out

    def scalars(self) -> dict:
        out = np.zeros(6, dtype=np.float64)
        lib().ora3_scalars(self._h, _dptr(out))
        d = dict(zip(["t", "dt", "smax", "step", "status", "dt_last"], out.tolist()))
        d["step"] = int(d["step"])
        d["status"] = int(d["status"])
        return d

    def close(self):
        if getattr(self, "_h", None):
            lib().ora3_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def run3(params: Params3, q0: np.ndarray, steps: int, t_end: float = -np.inf):
    """Convenience: run a 3D state and return (q, scalars)."""
    o = Oracle3(params, q0)
    o.run(steps, t_end)
    q, sc = o.q(), o.scalars()
    o.close()
    return q, sc


def interface3(beta: float, qL, qR):
    """One x1 interface of the 3D solver: (s[4], W[4,4] rows = families, amdq[4],
    apdq[4], nonreal)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    s, W, am, ap = np.zeros(4), np.zeros(16), np.zeros(4), np.zeros(4)
    nr = lib().ora3_interface(beta, _dptr(qL), _dptr(qR), _dptr(s), _dptr(W), _dptr(am),
                              _dptr(ap))
    return s, W.reshape(4, 4), am, ap, bool(nr)
