"""Build libdifvm.so (sm_103a) in-tree with nvcc.

The library is compiled for Blackwell Ultra only:
``-gencode arch=compute_103a,code=sm_103a``.  Each source file is compiled to
an object in parallel (no device code crosses files, so no relocatable device
code is needed) and the objects are linked into one shared library.  It links
the CUDA runtime dynamically so that it shares the runtime (and the primary
context) with PyTorch in the same process.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdifvm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]
LINK = ["-shared", "-cudart", "shared"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "difvm.h")]


def _deps():
    return sources() + _headers()


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def build(force: bool = False, verbose: bool = False, jobs: int = None) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    hdr_t = max(os.path.getmtime(p) for p in _headers())

    def compile_one(src):
        o = _obj(src)
        if (not force and os.path.exists(o)
                and os.path.getmtime(o) > max(os.path.getmtime(src), hdr_t)):
            return
        tmp = o + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", tmp, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, o)

    srcs = sources()
    with ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, *LINK, "-o", tmp, *[_obj(s) for s in srcs]]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
