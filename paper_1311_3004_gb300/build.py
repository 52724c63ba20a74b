"""Build the in-tree CUDA library libfvna.so for sm_103a.

The translation units are compiled in parallel with nvcc and linked with
the static CUDA runtime:
  fvna_fp64.cu  binary64 kernels, -fmad=false (products never fused into sums)
  fvna_fp32.cu  binary32 perturbation kernels
  fvna_api.cu   host runtime behind include/fvna.h
  fvna_noalloc.cu  the allocation-free binary64 step (fixed device scratch array)
  fvna_net.cu   the learned correction (BF16 tensor-core forward, FP32 backward)
  fvna_3d64.cu  the 3D step in binary64 (-fmad=false) and its dt bookkeeping
  fvna_3d32.cu  the 3D step in binary32 perturbation variables
  fvna_api3d.cu host runtime of the 3D entry points
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfvna.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
UNITS = {
    "fvna_fp64": ["-fmad=false"],
    "fvna_fp32": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "fvna_api": [],
    "fvna_noalloc": ["-fmad=false"],
    "fvna_net": [],
    "fvna_3d64": ["-fmad=false"],
    "fvna_3d32": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "fvna_api3d": [],
}


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)
            if f.endswith((".cu", ".cuh", ".h", ".inc"))] + \
           [os.path.join(os.path.dirname(HERE), "include", "fvna.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _compile(unit: str, verbose: bool) -> str:
    obj = os.path.join(OUT, unit + ".o")
    # FVNA_NVCC_FLAGS: extra flags (e.g. -DFVNA_MARCH_UNROLL=2) for tuning builds
    extra = os.environ.get("FVNA_NVCC_FLAGS", "").split()
    cmd = [NVCC, *ARCH, *COMMON, *UNITS[unit], *extra, "-c", os.path.join(CSRC, unit + ".cu"),
           "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale():
        return LIB
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
