"""Build libpint.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel into
_build/, then linked into paper_2504_02117_gb300/libpint.so. No cmake.
build(bounds=True) makes the checked variant libpint_bounds.so (objects in
_build_bounds/, -DPINT_BOUNDS: matrix index gathers are checked and a bad
index is recorded instead of used); the package loads it when the
environment variable PINT_LIB names it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpint.so")
BUILD_BOUNDS = os.path.join(PKG, "_build_bounds")
LIB_BOUNDS = os.path.join(PKG, "libpint_bounds.so")
SOURCES = ["api.cu", "spmm.cu", "krylov.cu", "ilu.cu", "fv.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra)


def _compile(src, extra, verbose, bdir=BUILD):
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(objs, lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(ROOT, "include", "pint.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra=(), bounds: bool = False) -> str:
    """Compile and link libpint.so (or, with bounds=True, the checked
    libpint_bounds.so); returns its path."""
    bdir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if bounds else (BUILD, LIB)
    extra = list(extra) + (["-DPINT_BOUNDS"] if bounds else [])
    os.makedirs(bdir, exist_ok=True)
    if not force and not _stale(None, lib):
        return lib
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, verbose, bdir), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, force="-f" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                bounds="--bounds" in sys.argv))
