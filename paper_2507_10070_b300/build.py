"""Build libann.so in-tree: CUDA sources for sm_103a with nvcc, host tooling
with g++ (float contraction off, so the PQ trainer's float64 arithmetic has a
fixed rounding order), linked into one shared library next to this file.

Usage: python -m paper_2507_10070_b300.build [--force]
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(ROOT, "_build", "libann")
LIB = os.path.join(PKG, "libann.so")
HEADERS = [os.path.join(ROOT, "include", "ann.h"), os.path.join(CSRC, "ann_internal.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-ffp-contract=off", "--expt-relaxed-constexpr"] + ARCH
CXX_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-ffp-contract=off", "-pthread", "-Wall"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libann")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, force: bool, extra=()) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(OBJ, src + ".o")
    if force or _stale(obj, [path] + HEADERS):
        if src.endswith(".cu"):
            cmd = [_nvcc(), *NVCC_FLAGS, *extra, "-c", path, "-o", obj]
        else:
            cmd = ["g++", *CXX_FLAGS, *extra, "-c", path, "-o", obj]
        subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile every source that changed and link libann.so; returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    extra = ("-Xptxas", "-v") if verbose_ptxas else ()
    srcs = _sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, extra if s.endswith(".cu") else ()), srcs))
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
