"""Builds liblbm.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2606_29619_b300.build [--force]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "liblbm.so")
MAIN = os.path.join(CSRC, "lbm_abi.cu")
UNITS = [MAIN, os.path.join(CSRC, "lbm_inplace.cu"), os.path.join(CSRC, "lbm_noalloc.cu")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "--expt-relaxed-constexpr",
    # FP32 division and square root by the fast hardware approximations; FP64 is unaffected
    "-prec-div=false", "-prec-sqrt=false", "-ftz=true",
]


def _sources():
    return UNITS + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "lbm.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the units in parallel (nvcc -c), then links the shared library."""
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    tag = f".tmp{os.getpid()}"
    objs, procs = [], []
    for u in UNITS:
        obj = os.path.join(PKG, os.path.splitext(os.path.basename(u))[0] + tag + ".o")
        cmd = [nvcc, *NVCC_FLAGS, *inc, "-c", "-o", obj, u]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        objs.append(obj)
        procs.append((u, subprocess.Popen(cmd)))
    failed = [u for u, pr in procs if pr.wait() != 0]
    try:
        if failed:
            raise subprocess.CalledProcessError(1, "nvcc -c " + " ".join(failed))
        tmp = LIB + tag
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
