"""Builds libsuperpoint.so and libspbounds.so in-tree with nvcc for sm_103a (GB300).

Each translation unit of csrc/ is compiled in parallel to an object under
_build/, then linked into paper_1901_07306_gb300/libsuperpoint.so (the C ABI
of include/superpoint.h); bounds/ holds the hardware probes of
include/sp_bounds.h, linked into paper_1901_07306_gb300/libspbounds.so.  The
CUDA runtime is linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BOUNDS = os.path.join(HERE, "bounds")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsuperpoint.so")
BOUNDS_LIB = os.path.join(HERE, "libspbounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden",
                     "-Xptxas", "-v"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsuperpoint")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _bounds_sources():
    return sorted(glob.glob(os.path.join(BOUNDS, "*.cu")))


def _deps():
    inc = os.path.join(os.path.dirname(HERE), "include")
    return (_sources() + _bounds_sources() + sorted(glob.glob(os.path.join(CSRC, "*.h"))) +
            sorted(glob.glob(os.path.join(inc, "*.h"))) + [os.path.abspath(__file__)])


def _stale() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(BOUNDS_LIB)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(BOUNDS_LIB))
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources() + _bounds_sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        log = os.path.join(BUILD, os.path.basename(src) + ".log")
        with open(log, "w") as f:
            f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr[-4000:]}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    n_main = len(_sources())
    for lib, parts in ((LIB, objs[:n_main]), (BOUNDS_LIB, objs[n_main:])):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *parts], check=True, capture_output=not verbose)
        os.replace(tmp, lib)
    if verbose:
        for log in sorted(glob.glob(os.path.join(BUILD, "*.log"))):
            sys.stdout.write(open(log).read())
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
