"""The C-ABI library loads, exports every function include/fvna.h declares,
its struct layouts match the Python mirrors, and argument checks fire before
any device work (no GPU needed for any of this)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1311_3004_gb300 import build as fbuild
from paper_1311_3004_gb300 import fvna

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fvna.h")


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fvna.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fvna_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", fvna.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (fvna_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "fvna.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("fvna_config %zu\nfvna_domain %zu\nfvna_stats %zu\nfvna_domain3 %zu\n",
         sizeof(fvna_config), sizeof(fvna_domain), sizeof(fvna_stats), sizeof(fvna_domain3));
  P(fvna_config, beta); P(fvna_config, dt_fixed); P(fvna_config, tile_y);
  P(fvna_config, compensated); P(fvna_config, splitting);
  P(fvna_domain, x0); P(fvna_domain, dt0); P(fvna_domain, aperture);
  P(fvna_stats, nu_std); P(fvna_stats, status);
  P(fvna_config, wait_limit);
  P(fvna_domain3, nz); P(fvna_domain3, bc); P(fvna_domain3, substeps); P(fvna_domain3, t0);
  P(fvna_domain3, dt0);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "probe.c")
        exe = os.path.join(td, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    assert int(got["fvna_config"]) == ctypes.sizeof(fvna.Config)
    assert int(got["fvna_domain"]) == ctypes.sizeof(fvna.Domain)
    assert int(got["fvna_stats"]) == ctypes.sizeof(fvna.Stats)
    assert int(got["fvna_domain3"]) == ctypes.sizeof(fvna.Domain3)
    for key, v in got.items():
        if "." in key:
            T, f = key.split(".")
            cls = {"fvna_config": fvna.Config, "fvna_domain": fvna.Domain,
                   "fvna_stats": fvna.Stats, "fvna_domain3": fvna.Domain3}[T]
            assert getattr(cls, f).offset == int(v), key


def _init(cfg, doms, q0s):
    L = fvna.lib()
    n = len(doms)
    darr = (fvna.Domain * n)(*doms) if n else None
    ptrs = (ctypes.c_void_p * max(n, 1))(*[q.ctypes.data for q in q0s])
    h = ctypes.c_void_p()
    rc = L.fvna_init(ctypes.byref(cfg) if cfg is not None else None, n, darr, ptrs, 0, None,
                     ctypes.byref(h))
    return rc, h


def test_argument_errors_before_device_work(lib):
    import numpy as np
    q = np.zeros((3, 4, 4))
    q[0] = 1.0
    good = fvna.make_config()
    dom = fvna.make_domain(4, 4)
    bad_cfgs = [
        fvna.make_config(precision=7), fvna.make_config(geometry=3), fvna.make_config(limiter=9),
        fvna.make_config(sweeps=8), fvna.make_config(dx=0.0), fvna.make_config(dx=-1.0),
        fvna.make_config(nu_w=0.0), fvna.make_config(nu_max=0.0), fvna.make_config(delta=-1.0),
        fvna.make_config(tile_x=48), fvna.make_config(tile_x=8), fvna.make_config(tile_y=4),
        fvna.make_config(steps_per_graph=-1), fvna.make_config(compensated=2),
    ]
    for cfg in bad_cfgs:
        rc, h = _init(cfg, [dom], [q])
        assert rc == fvna.ERR_ARG and not h.value
    bad_doms = [
        fvna.make_domain(0, 4), fvna.make_domain(4, 0), fvna.make_domain(4, 4, bc=(9, 1, 1, 1)),
        fvna.make_domain(2, 4, bc=(fvna.BC_PERIODIC, fvna.BC_PERIODIC, 1, 1)),
        fvna.make_domain(4, 2, bc=(1, 1, fvna.BC_REFLECT, 1)),
        fvna.make_domain(4, 4, bc=(fvna.BC_PERIODIC, fvna.BC_EXTRAP, 1, 1)),
        fvna.make_domain(4, 4, bc=(fvna.BC_HIFU, 1, 1, 1), focal=0.0),
        fvna.make_domain(4, 4, dt0=-1.0),
    ]
    for d in bad_doms:
        rc, h = _init(good, [d], [q])
        assert rc == fvna.ERR_ARG and not h.value
    rc, h = _init(None, [dom], [q])
    assert rc == fvna.ERR_ARG
    rc, h = _init(good, [], [])
    assert rc == fvna.ERR_ARG
    # the other entry points reject NULL contexts and bad arguments
    assert lib.fvna_step(None, 1) == fvna.ERR_ARG
    assert lib.fvna_run(None, 1.0, 1, None) == fvna.ERR_ARG
    assert lib.fvna_sync(None) == fvna.ERR_ARG
    assert lib.fvna_fields(None, 0, 0, None, 0, 0) == fvna.ERR_ARG
    assert lib.fvna_launch_count(None) == 0
    assert lib.fvna_step_timed(None, None) == fvna.ERR_ARG
    assert lib.fvna_shift(None, 0, 1, 0) == fvna.ERR_ARG
    assert lib.fvna_set_bc(None, 0, 0, fvna.BC_EXTRAP) == fvna.ERR_ARG
    assert lib.fvna_run_moving(None, 1.0, 1, 0.0, 1.0, 0.0, 1, None) == fvna.ERR_ARG
    lib.fvna_destroy(None)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.fvna_riemann(5, 3.5, 1, None, None, None, None, None, None) == fvna.ERR_ARG
    assert lib.fvna_riemann(0, 3.5, -1, None, None, None, None, None, None) == fvna.ERR_ARG
    assert lib.fvna_riemann(0, 3.5, 0, None, None, None, None, None, None) == fvna.OK
    for code in [0, -1, -2, -3, -4, -5, -6, -7]:
        assert lib.fvna_strerror(code)
    assert b"unknown" in lib.fvna_strerror(-99)


def test_step_noalloc_refuses_wrong_buffers_before_any_launch(lib):
    """fvna_step_noalloc takes bare device pointers, so the binding checks the
    buffers' type, layout and size itself and raises before the C call."""
    torch = pytest.importorskip("torch")
    cfg = fvna.make_config(precision=fvna.FP64, dx=0.1, dt_fixed=0.01)
    dom = fvna.make_domain(8, 5)
    good = torch.zeros((3, 5, 8), dtype=torch.float64)
    bad = [torch.zeros((3, 5, 8), dtype=torch.float32),              # binary32
           torch.zeros((3, 5, 7), dtype=torch.float64),              # too small
           torch.zeros((3, 8, 5), dtype=torch.float64).transpose(1, 2),  # not contiguous
           good.numpy(),                                             # not a tensor
           good]                                                     # host memory
    for b in bad:
        with pytest.raises(fvna.FvnaError) as e:
            fvna.step_noalloc(cfg, dom, b, b, 0.0, 0.01)
        assert e.value.code == fvna.ERR_ARG
