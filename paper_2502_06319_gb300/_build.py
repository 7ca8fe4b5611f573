"""Build libcosmica.so in-tree with nvcc for sm_103a (GB300).

Each translation unit gets the floating-point flags its arithmetic needs:
  * k_fp64.cu, k_spectrum.cu: -fmad=false -- FP64 expressions evaluated exactly
    as written (no FMA contraction), so the FP64 path is reproducible bit for bit;
  * k_mixed.cu, k_serve.cu, k_debug32.cu: -ftz=true -prec-div=false -prec-sqrt=false
    -fmad=false -- the mixed path deliberately uses the SFU approximations, and
    writes every FMA explicitly so that its rounding is the same in every
    kernel and inlining context;
  * cosmica_api.cu, server.cu, k_noalloc.cu, k_debug_curand.cu: defaults.
Objects are compiled in parallel and linked into one shared library next to
this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcosmica.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
# the mixed path: flush-to-zero, approximate division and square root (it uses
# the SFU intrinsics deliberately), and no automatic FMA contraction -- every
# FMA of the step is written out, so its rounding cannot depend on context
MIXED_FLAGS = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false", "-fmad=false"]
UNITS = {
    "cosmica_api.cu": [],
    "k_fp64.cu": ["-fmad=false"],
    "k_spectrum.cu": ["-fmad=false"],
    "k_mixed.cu": MIXED_FLAGS,
    "k_serve.cu": MIXED_FLAGS,
    "server.cu": [],
    "k_noalloc.cu": [],
    "k_debug_curand.cu": [],
    "k_debug32.cu": MIXED_FLAGS,
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcosmica")


def _sources_mtime() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return max(t, os.path.getmtime(__file__))


def _compile(unit: str, flags, verbose: bool) -> str:
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    cmd = [nvcc()] + COMMON + flags + (["-Xptxas", "-v"] if verbose else []) + \
        ["-c", os.path.join(CSRC, unit), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libcosmica.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose), UNITS.items()))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
