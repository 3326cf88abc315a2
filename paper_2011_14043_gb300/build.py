"""Compile the CUDA library (sm_103a) in-tree: ``_build/libfdtd.so``.

Two translation units, one ``-gencode``; takes about ten seconds.  The
library links the CUDA runtime statically, so it only needs the driver at
run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libfdtd.so")
# the bounds-checked debug build (-DFDTD_BOUNDS): every kernel line, tile or
# element range is checked against its array's extent (FDTD_ERR_BOUNDS)
BOUNDS_LIB_PATH = os.path.join(BUILD_DIR, "libfdtd_bounds.so")
SOURCES = [os.path.join(HERE, "csrc", "fdtd.cu"), os.path.join(HERE, "csrc", "energy_noalloc.cu")]
DEPENDS = SOURCES + [
    os.path.join(HERE, "csrc", "line_kernels.cuh"),
    os.path.join(HERE, "csrc", "aux_kernels.cuh"),
    os.path.join(HERE, "csrc", "adjoint_kernels.cuh"),
    os.path.join(HERE, "csrc", "line4_kernels.cuh"),
    os.path.join(ROOT, "include", "fdtd.h"),
]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"),
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
                 shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set CUDA_HOME or NVCC)")


def up_to_date(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return False
    t = os.path.getmtime(path)
    return all(os.path.getmtime(p) <= t for p in DEPENDS)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Build ``libfdtd.so`` (or, with bounds, the bounds-checked
    ``libfdtd_bounds.so``) if missing or stale; returns its path."""
    path = BOUNDS_LIB_PATH if bounds else LIB_PATH
    if not force and up_to_date(path):
        return path
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = path + ".tmp"
    cmd = [nvcc_path(), ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
           "-shared", "-o", tmp] + (["-DFDTD_BOUNDS"] if bounds else []) + SOURCES
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stdout + res.stderr)
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(build(force=True))
