"""Python binding of the C ABI in include/fvna.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of libfvna.so; this module
converts arguments and raises FvnaError on a nonzero status.  If the library
has not been built the import of `lib()` fails loudly: there is no CPU path.

PyTorch serves only as the source of device memory and of the current CUDA
stream when the caller passes torch tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfvna.so")

FP64, FP32_PERT = 0, 1
CARTESIAN, AXISYMMETRIC = 0, 1
LIM_MC, LIM_NONE, LIM_LW = 0, 1, 2
SPLIT_GODUNOV, SPLIT_STRANG = 0, 1
BC_PERIODIC, BC_EXTRAP, BC_REFLECT, BC_TAYLOR, BC_HIFU = 0, 1, 2, 3, 4
FIELD_Q, FIELD_PRESSURE, FIELD_BUDGET, FIELD_STATS, FIELD_CORNER, FIELD_AXIS = 0, 1, 2, 3, 4, 5
FIELD_OUTFLOW = 6

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NONREAL, ERR_CFL, ERR_NAN = 0, -1, -2, -3, -4, -5, -6
ERR_SIZE = -7
ERR_TIMEOUT = -8
NOALLOC_MAX_CELLS = 524288


class FvnaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if code in (ERR_CUDA, ERR_OOM):
            msg += f" [{lib().fvna_last_cuda_error().decode()}]"
        super().__init__(msg)


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("geometry", ctypes.c_int),
                ("limiter", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("beta", ctypes.c_double), ("delta", ctypes.c_double), ("dx", ctypes.c_double),
                ("nu_w", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("steps_per_graph", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("compensated", ctypes.c_int),
                ("splitting", ctypes.c_int), ("wait_limit", ctypes.c_int)]


class Domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("envelope", ctypes.c_int), ("reserved", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("t0", ctypes.c_double),
                ("dt0", ctypes.c_double), ("taylor_ratio", ctypes.c_double), ("taylor_angle", ctypes.c_double),
                ("amp", ctypes.c_double), ("focal", ctypes.c_double),
                ("aperture", ctypes.c_double)]


class Domain3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 6), ("substeps", ctypes.c_int),
                ("t0", ctypes.c_double), ("dt0", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("dt_last", ctypes.c_double), ("smax", ctypes.c_double),
                ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("nu_mean", ctypes.c_double), ("nu_std", ctypes.c_double),
                ("status", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "reserved"}


SYMBOLS = ["fvna_init", "fvna_step", "fvna_run", "fvna_sync", "fvna_fields",
           "fvna_step_timed", "fvna_launch_count", "fvna_destroy", "fvna_strerror", "fvna_riemann",
           "fvna_last_cuda_error",
           "fvna_step_noalloc", "fvna_autotune", "fvna_net_create", "fvna_net_params",
           "fvna_net_forward", "fvna_net_backward", "fvna_net_train_step", "fvna_net_destroy",
           "fvna_set_correction", "fvna_set_budgets", "fvna3_init", "fvna3_run", "fvna3_step_timed", "fvna3_fields",
           "fvna3_launch_count", "fvna3_destroy"]

_lib = None


def lib():
    """Load libfvna.so (raises if it was not built: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run __graft_entry__.build() or "
                          "python -m paper_1311_3004_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.fvna_init.restype = ctypes.c_int
    L.fvna_init.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(Domain),
                            ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, vp,
                            ctypes.POINTER(vp)]
    L.fvna_step.restype = ctypes.c_int
    L.fvna_step.argtypes = [vp, ctypes.c_longlong]
    L.fvna_run.restype = ctypes.c_int
    L.fvna_run.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(Stats)]
    L.fvna_shift.restype = ctypes.c_int
    L.fvna_shift.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fvna_set_bc.restype = ctypes.c_int
    L.fvna_set_bc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fvna_run_moving.restype = ctypes.c_int
    L.fvna_run_moving.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(Stats)]
    L.fvna_sync.restype = ctypes.c_int
    L.fvna_sync.argtypes = [vp]
    L.fvna_fields.restype = ctypes.c_int
    L.fvna_fields.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
    L.fvna_step_timed.restype = ctypes.c_int
    L.fvna_step_timed.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.fvna_launch_count.restype = ctypes.c_longlong
    L.fvna_launch_count.argtypes = [vp]
    L.fvna_destroy.restype = None
    L.fvna_destroy.argtypes = [vp]
    L.fvna_strerror.restype = ctypes.c_char_p
    L.fvna_strerror.argtypes = [ctypes.c_int]
    L.fvna_last_cuda_error.restype = ctypes.c_char_p
    L.fvna_last_cuda_error.argtypes = []
    L.fvna_autotune.restype = ctypes.c_int
    L.fvna_autotune.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(Domain),
                                ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, vp, ctypes.c_int,
                                ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_float)]
    L.fvna_net_create.restype = ctypes.c_int
    L.fvna_net_create.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(vp)]
    L.fvna_net_params.restype = ctypes.c_int
    L.fvna_net_params.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    L.fvna_net_forward.restype = ctypes.c_int
    L.fvna_net_forward.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                   ctypes.c_float, vp, vp, vp, vp]
    L.fvna_net_backward.restype = ctypes.c_int
    L.fvna_net_backward.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                    ctypes.c_float, vp, vp, vp]
    L.fvna_net_train_step.restype = ctypes.c_int
    L.fvna_net_train_step.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                      ctypes.c_float, vp, ctypes.c_int, vp, ctypes.c_float,
                                      ctypes.POINTER(ctypes.c_double), vp]
    L.fvna_net_destroy.restype = None
    L.fvna_net_destroy.argtypes = [vp]
    L.fvna_set_correction.restype = ctypes.c_int
    L.fvna_set_correction.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                      ctypes.c_int]
    L.fvna_step_noalloc.restype = ctypes.c_int
    L.fvna_step_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Domain), vp, vp,
                                    ctypes.c_double, ctypes.c_double, dp, vp]
    L.fvna_set_budgets.restype = ctypes.c_int
    L.fvna_set_budgets.argtypes = [vp, ctypes.c_int]
    L.fvna3_init.restype = ctypes.c_int
    L.fvna3_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Domain3), vp, ctypes.c_int, vp,
                             ctypes.POINTER(vp)]
    L.fvna3_run.restype = ctypes.c_int
    L.fvna3_run.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(Stats)]
    L.fvna3_step_timed.restype = ctypes.c_int
    L.fvna3_step_timed.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.fvna3_fields.restype = ctypes.c_int
    L.fvna3_fields.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
    L.fvna3_launch_count.restype = ctypes.c_longlong
    L.fvna3_launch_count.argtypes = [vp]
    L.fvna3_destroy.restype = None
    L.fvna3_destroy.argtypes = [vp]
    L.fvna_riemann.restype = ctypes.c_int
    L.fvna_riemann.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp, dp]
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().fvna_strerror(code).decode()
    except ImportError:
        return f"status {code}"


def _check(rc: int, where: str) -> int:
    if rc != OK:
        raise FvnaError(rc, where)
    return rc


def make_config(precision=FP64, geometry=CARTESIAN, limiter=LIM_MC, sweeps=7, beta=3.5,
                delta=0.0, dx=1.0, nu_w=0.9, nu_max=1.0, dt_fixed=0.0, steps_per_graph=0,
                tile_x=0, tile_y=0, compensated=0, splitting=0, wait_limit=0) -> Config:
    return Config(precision, geometry, limiter, sweeps, beta, delta, dx, nu_w, nu_max, dt_fixed,
                  steps_per_graph, tile_x, tile_y, compensated, splitting, wait_limit)


def make_domain(nx, ny, bc=(BC_EXTRAP,) * 4, envelope=0, x0=0.0, y0=0.0, t0=0.0, dt0=0.0,
                taylor_ratio=0.0, taylor_angle=0.0, amp=0.0, focal=1.0, aperture=0.0) -> Domain:
    return Domain(nx, ny, (ctypes.c_int * 4)(*bc), envelope, 0, x0, y0, t0, dt0, taylor_ratio,
                  taylor_angle, amp, focal, aperture)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _marshal_states(domains, q0):
    """Pointers to the initial states (numpy host arrays or torch CUDA tensors)."""
    n = len(domains)
    on_dev = False
    keep = []
    ptrs = (ctypes.c_void_p * n)()
    for i, (d, q) in enumerate(zip(domains, q0)):
        if hasattr(q, "is_cuda") and q.is_cuda:
            import torch
            q = q.to(torch.float64).contiguous()
            assert tuple(q.shape) == (3, d.ny, d.nx)
            on_dev = True
            ptrs[i] = q.data_ptr()
        else:
            q = np.ascontiguousarray(q, dtype=np.float64)
            assert q.shape == (3, d.ny, d.nx), (q.shape, d.ny, d.nx)
            ptrs[i] = q.ctypes.data
        keep.append(q)
    return ptrs, on_dev, keep


def autotune(config: Config, domains: Sequence[Domain], q0: Sequence, trial_steps: int = 8,
             stream=None):
    """Fastest sweep tile shapes for these domains (fvna_autotune): (Config, ms/step)."""
    ptrs, on_dev, keep = _marshal_states(domains, q0)
    if stream is None:
        stream = _current_stream()
    n = len(domains)
    darr = (Domain * n)(*domains)
    best = Config()
    ms = ctypes.c_float(0.0)
    _check(lib().fvna_autotune(ctypes.byref(config), n, darr, ptrs, int(on_dev),
                               ctypes.c_void_p(stream), int(trial_steps), ctypes.byref(best),
                               ctypes.byref(ms)), "fvna_autotune")
    return best, float(ms.value)


def make_domain3(nx, ny, nz, bc=(BC_EXTRAP,) * 6, t0=0.0, dt0=0.0, substeps=0) -> Domain3:
    """substeps: 0 the full step, else bit 0 x1, bit 1 x2, bit 2 x3, bit 3 source."""
    return Domain3(nx, ny, nz, (ctypes.c_int * 6)(*bc), substeps, t0, dt0)


class Solver3:
    """One 3D domain (fvna3_*).  q0: (4, nz, ny, nx) binary64 total variables,
    a numpy array (host) or a torch CUDA tensor (device).  domain.substeps
    selects sub-steps (0: the full step)."""

    def __init__(self, config: Config, domain: Domain3, q0, stream=None):
        L = lib()
        self.config = config
        self.domain = domain
        shape = (4, domain.nz, domain.ny, domain.nx)
        if hasattr(q0, "is_cuda") and q0.is_cuda:
            import torch
            q = q0.to(torch.float64).contiguous()
            on_dev, ptr = 1, q.data_ptr()
        else:
            q = np.ascontiguousarray(q0, dtype=np.float64)
            on_dev, ptr = 0, q.ctypes.data
        assert tuple(q.shape) == shape, (tuple(q.shape), shape)
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(L.fvna3_init(ctypes.byref(config), ctypes.byref(domain), ctypes.c_void_p(ptr),
                            on_dev, ctypes.c_void_p(stream), ctypes.byref(h)), "fvna3_init")
        self._h = h

    def run(self, t_end: float = -np.inf, max_steps: int = 2 ** 62, check: bool = True) -> dict:
        st = Stats()
        t_end = float(t_end) if np.isfinite(t_end) else -1e300
        rc = lib().fvna3_run(self._h, t_end, int(max_steps), ctypes.byref(st))
        if check:
            _check(rc, "fvna3_run")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def step_timed(self):
        """One step with per-kernel device times (ms): x1, x2, x3 sweeps, source, dt update."""
        ms = (ctypes.c_float * 5)()
        _check(lib().fvna3_step_timed(self._h, ms), "fvna3_step_timed")
        return tuple(float(x) for x in ms)

    def q(self, out=None):
        """State as (4, nz, ny, nx) binary64 (numpy, or into a torch CUDA tensor)."""
        d = self.domain
        n = 4 * d.nx * d.ny * d.nz
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            _check(lib().fvna3_fields(self._h, FIELD_Q, ctypes.c_void_p(out.data_ptr()),
                                      out.numel() * out.element_size(), 1), "fvna3_fields")
            return out
        q = np.empty((4, d.nz, d.ny, d.nx), dtype=np.float64)
        _check(lib().fvna3_fields(self._h, FIELD_Q, q.ctypes.data_as(ctypes.c_void_p), n * 8, 0),
               "fvna3_fields")
        return q

    def stats(self) -> dict:
        st = Stats()
        _check(lib().fvna3_fields(self._h, FIELD_STATS, ctypes.cast(ctypes.byref(st),
                                                                    ctypes.c_void_p),
                                  ctypes.sizeof(st), 0), "fvna3_fields")
        return st.as_dict()

    def launch_count(self) -> int:
        return int(lib().fvna3_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().fvna3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """A context of one or more domains advancing together.

    q0: one array per domain of shape (3, ny, nx), binary64 total variables;
    numpy arrays (host) or torch CUDA tensors (device), not mixed.
    """

    def __init__(self, config: Config, domains: Sequence[Domain], q0: Sequence, stream=None):
        L = lib()
        self.config = config
        self.domains = list(domains)
        n = len(self.domains)
        ptrs, on_dev, keep = _marshal_states(self.domains, q0)
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        darr = (Domain * n)(*self.domains)
        h = ctypes.c_void_p()
        _check(L.fvna_init(ctypes.byref(config), n, darr, ptrs, int(on_dev),
                           ctypes.c_void_p(stream), ctypes.byref(h)), "fvna_init")
        self._h = h

    # -- stepping -----------------------------------------------------------
    def step(self, nsteps: int) -> None:
        _check(lib().fvna_step(self._h, int(nsteps)), "fvna_step")

    def run(self, t_end: float = -np.inf, max_steps: int = 2 ** 62, check: bool = True) -> dict:
        st = Stats()
        t_end = float(t_end) if np.isfinite(t_end) else -1e300
        rc = lib().fvna_run(self._h, t_end, int(max_steps), ctypes.byref(st))
        if check:
            _check(rc, "fvna_run")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def shift(self, domain: int, kx: int, ky: int) -> None:
        """Move the window of one domain by (kx, ky) cells (fvna_shift)."""
        _check(lib().fvna_shift(self._h, int(domain), int(kx), int(ky)), "fvna_shift")

    def set_bc(self, domain: int, side: int, bc: int) -> None:
        """Change the border rule of one side between steps (fvna_set_bc)."""
        _check(lib().fvna_set_bc(self._h, int(domain), int(side), int(bc)), "fvna_set_bc")

    def run_moving(self, t_end: float, t1: float, velocity, every: int,
                   max_steps: int = 2 ** 62, check: bool = True) -> dict:
        """Two-stage run: windows at rest until t1, then moving at `velocity` (fvna_run_moving)."""
        st = Stats()
        t_end = float(t_end) if np.isfinite(t_end) else -1e300
        rc = lib().fvna_run_moving(self._h, t_end, int(max_steps), float(t1), float(velocity[0]),
                                   float(velocity[1]), int(every), ctypes.byref(st))
        if check:
            _check(rc, "fvna_run_moving")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def step_timed(self):
        """One step with per-kernel device times (ms): (x1 sweep, x2 sweep + source, dt update)."""
        ms = (ctypes.c_float * 3)()
        _check(lib().fvna_step_timed(self._h, ms), "fvna_step_timed")
        return float(ms[0]), float(ms[1]), float(ms[2])

    def sync(self) -> int:
        return lib().fvna_sync(self._h)

    # -- outputs ------------------------------------------------------------
    def q(self, domain: int = 0, out=None):
        """State of one domain as (3, ny, nx) binary64 (numpy, or into a torch CUDA tensor)."""
        d = self.domains[domain]
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            _check(lib().fvna_fields(self._h, domain, FIELD_Q, ctypes.c_void_p(out.data_ptr()),
                                     out.numel() * out.element_size(), 1), "fvna_fields")
            return out
        arr = np.empty((3, d.ny, d.nx), dtype=np.float64) if out is None else out
        _check(lib().fvna_fields(self._h, domain, FIELD_Q, ctypes.c_void_p(arr.ctypes.data),
                                 arr.nbytes, 0), "fvna_fields")
        return arr

    def pressure(self, domain: int = 0):
        d = self.domains[domain]
        arr = np.empty((d.ny, d.nx), dtype=np.float64)
        _check(lib().fvna_fields(self._h, domain, FIELD_PRESSURE, ctypes.c_void_p(arr.ctypes.data),
                                 arr.nbytes, 0), "fvna_fields")
        return arr

    def axis_pressure(self, domain: int = 0):
        """p'/(rho0 c0^2) along row 0 (nx values)."""
        d = self.domains[domain]
        arr = np.empty(d.nx, dtype=np.float64)
        _check(lib().fvna_fields(self._h, domain, FIELD_AXIS, ctypes.c_void_p(arr.ctypes.data),
                                 arr.nbytes, 0), "fvna_fields")
        return arr

    def budget(self, domain: int = 0):
        arr = np.zeros(3, dtype=np.float64)
        _check(lib().fvna_fields(self._h, domain, FIELD_BUDGET, ctypes.c_void_p(arr.ctypes.data),
                                 arr.nbytes, 0), "fvna_fields")
        return arr

    def set_budgets(self, on: bool = True) -> None:
        """Per-step boundary-flux budget on or off (fvna_set_budgets; on resets it)."""
        _check(lib().fvna_set_budgets(self._h, int(bool(on))), "fvna_set_budgets")

    def outflow(self, domain: int = 0):
        """Boundary-flux budget of (q1, q2, q3) since it was switched on."""
        arr = np.zeros(3, dtype=np.float64)
        _check(lib().fvna_fields(self._h, domain, FIELD_OUTFLOW,
                                 ctypes.c_void_p(arr.ctypes.data), arr.nbytes, 0), "fvna_fields")
        return arr

    def corner(self, domain: int = 0):
        """Lower-left corner (x0, y0) of the domain's window."""
        arr = np.zeros(2, dtype=np.float64)
        _check(lib().fvna_fields(self._h, domain, FIELD_CORNER, ctypes.c_void_p(arr.ctypes.data),
                                 arr.nbytes, 0), "fvna_fields")
        return float(arr[0]), float(arr[1])

    def stats(self, domain: int = 0) -> dict:
        st = Stats()
        _check(lib().fvna_fields(self._h, domain, FIELD_STATS, ctypes.cast(ctypes.byref(st),
                                 ctypes.c_void_p), ctypes.sizeof(st), 0), "fvna_fields")
        return st.as_dict()

    def launch_count(self) -> int:
        return int(lib().fvna_launch_count(self._h))

    def set_correction(self, net, in_scale: float, out_scale: float, every: int = 1,
                       edge_band: int = 0) -> None:
        """Add out_scale * net(in_scale * state) after every `every`-th step,
        except within edge_band cells of the domain edges (net=None detaches)."""
        self._net = net
        _check(lib().fvna_set_correction(self._h, net._h if net is not None else None,
                                         float(in_scale), float(out_scale), int(every),
                                         int(edge_band)),
               "fvna_set_correction")

    def close(self):
        if getattr(self, "_h", None):
            lib().fvna_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NET_PARAMS = 11011


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Net:
    """The learned correction network (fvna_net_*): torch CUDA tensors in and
    out, all arithmetic in the library's kernels."""

    def __init__(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        assert p.size == NET_PARAMS
        h = ctypes.c_void_p()
        _check(lib().fvna_net_create(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     ctypes.byref(h)), "fvna_net_create")
        self._h = h

    def params(self) -> np.ndarray:
        out = np.zeros(NET_PARAMS, dtype=np.float32)
        _check(lib().fvna_net_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     None), "fvna_net_params")
        return out

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        _check(lib().fvna_net_params(self._h, None,
                                     p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "fvna_net_params")

    def forward(self, x, in_scale: float = 1.0, hidden: bool = False, stream=None):
        """x: (B, 3, h, w) float32 CUDA tensor -> y (and the two bf16 hidden
        activations as int16 bit patterns (B, h, w, 32) if hidden)."""
        import torch
        B, C, H, W = x.shape
        y = torch.empty_like(x)
        h1 = h2 = None
        if hidden:
            h1 = torch.empty((B, H, W, 32), dtype=torch.int16, device=x.device)
            h2 = torch.empty_like(h1)
        _check(lib().fvna_net_forward(self._h, B, H, W, _ptr(x), float(in_scale), _ptr(y),
                                      _ptr(h1), _ptr(h2),
                                      ctypes.c_void_p(stream or _current_stream())),
               "fvna_net_forward")
        return (y, h1, h2) if hidden else y

    def backward(self, x, gy, in_scale: float = 1.0, stream=None):
        import torch
        B, C, H, W = x.shape
        g = torch.empty(NET_PARAMS, dtype=torch.float32, device=x.device)
        _check(lib().fvna_net_backward(self._h, B, H, W, _ptr(x), float(in_scale), _ptr(gy),
                                       _ptr(g), ctypes.c_void_p(stream or _current_stream())),
               "fvna_net_backward")
        return g

    def train_step(self, x, target, lr: float, in_scale: float = 1.0, margin: int = 0,
                   edges=None, stream=None) -> float:
        """edges: optional int32 CUDA tensor (B, 4) of per-side margins."""
        B, C, H, W = x.shape
        loss = ctypes.c_double(0.0)
        _check(lib().fvna_net_train_step(self._h, B, H, W, _ptr(x), float(in_scale), _ptr(target),
                                         int(margin), _ptr(edges), float(lr), ctypes.byref(loss),
                                         ctypes.c_void_p(stream or _current_stream())),
               "fvna_net_train_step")
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fvna_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_params_flat(p: dict) -> np.ndarray:
    """Flatten a parameter dict (w1 b1 w2 b2 w3 b3, [out][in][row][col]) to the ABI layout."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1)
                           for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def net_params_dict(flat: np.ndarray) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    shapes = [("w1", (32, 3, 3, 3)), ("b1", (32,)), ("w2", (32, 32, 3, 3)), ("b2", (32,)),
              ("w3", (3, 32, 3, 3)), ("b3", (3,))]
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = flat[o:o + n].reshape(sh)
        o += n
    return out


def _check_noalloc_buffers(domain: Domain, *bufs) -> None:
    import torch
    n = 3 * int(domain.nx) * int(domain.ny)
    for b in bufs:
        if not isinstance(b, torch.Tensor):
            raise FvnaError(ERR_ARG, "step_noalloc: buffers must be torch tensors")
        if b.dtype != torch.float64:
            raise FvnaError(ERR_ARG, f"step_noalloc: buffer dtype {b.dtype}, expected float64")
        if not b.is_contiguous():
            raise FvnaError(ERR_ARG, "step_noalloc: buffer is not contiguous")
        if b.numel() != n:
            raise FvnaError(ERR_ARG, f"step_noalloc: buffer holds {b.numel()} values, the "
                                     f"domain needs 3*nx*ny = {n}")
        if not b.is_cuda or b.device.index != torch.cuda.current_device():
            raise FvnaError(ERR_ARG, f"step_noalloc: buffer on {b.device}, expected the "
                                     "current CUDA device")


def step_noalloc(config: Config, domain: Domain, q_in, q_out, t: float, dt: float,
                 stream=None):
    """One binary64 step that allocates nothing (fvna_step_noalloc).

    q_in, q_out: torch CUDA float64 tensors of shape (3, ny, nx) owned by the
    caller (they may be the same tensor).  Returns (status, max|s|).  The C
    entry point takes bare device pointers and cannot see a buffer's type or
    size, so a wrong tensor is refused here (FvnaError, ERR_ARG) before
    anything is launched."""
    _check_noalloc_buffers(domain, q_in, q_out)
    if stream is None:
        stream = _current_stream()
    sm = ctypes.c_double(0.0)
    rc = lib().fvna_step_noalloc(ctypes.byref(config), ctypes.byref(domain),
                                 ctypes.c_void_p(q_in.data_ptr()),
                                 ctypes.c_void_p(q_out.data_ptr()), float(t), float(dt),
                                 ctypes.byref(sm), ctypes.c_void_p(stream))
    return rc, sm.value


def riemann(precision: int, beta: float, qL, qR):
    """Device Roe solver on n pairs of cells (n, 3): returns s (n,3), W (n,3,3),
    amdq (n,3), apdq (n,3), nonreal flag."""
    qL = np.ascontiguousarray(qL, dtype=np.float64).reshape(-1, 3)
    qR = np.ascontiguousarray(qR, dtype=np.float64).reshape(-1, 3)
    n = qL.shape[0]
    s = np.zeros((n, 3))
    W = np.zeros((n, 3, 3))
    am = np.zeros((n, 3))
    ap = np.zeros((n, 3))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().fvna_riemann(precision, beta, n, qL.ctypes.data_as(dp), qR.ctypes.data_as(dp),
                            s.ctypes.data_as(dp), W.ctypes.data_as(dp), am.ctypes.data_as(dp),
                            ap.ctypes.data_as(dp))
    if rc not in (OK, ERR_NONREAL):
        raise FvnaError(rc, "fvna_riemann")
    return s, W, am, ap, rc == ERR_NONREAL
