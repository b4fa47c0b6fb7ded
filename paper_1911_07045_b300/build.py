"""Build ``liblqmin.so`` (the C-ABI library) in-tree with nvcc for sm_103a.

Usage: ``python -m paper_1911_07045_b300.build [--verbose]``.  The library
is rebuilt only when a source or header is newer than it.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblqmin.so")
LIB_BOUNDS = os.path.join(HERE, "liblqmin_bounds.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "lqmin.h")])


def needs_build(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Build ``liblqmin.so``; with ``bounds_check`` the bounds-checked
    variant ``liblqmin_bounds.so`` (every index of the step kernels checked
    and counted, see lq_bounds_check_hits) for the tests."""
    lib = LIB_BOUNDS if bounds_check else LIB
    if not force and not needs_build(lib):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
           "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
           "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *sources()]
    if bounds_check:
        cmd.insert(1, "-DLQ_BOUNDS_CHECK")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
