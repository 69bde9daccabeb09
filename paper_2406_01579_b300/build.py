"""Builds libtets.so (the CUDA kernels + C ABI) in the package directory for
sm_103a with nvcc.  Run ``python -m paper_2406_01579_b300.build``."""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libtets.so")
SOURCES = ["bin.cu", "blend.cu", "api.cu", "sort_noalloc.cu", "regularize.cu", "marching.cu"]
# ALU peak microbenchmarks for the roofline (a library of their own)
PEAKS_LIB = os.path.join(HERE, "libtets_peaks.so")
PEAKS_SOURCE = "peaks.cu"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _deps():
    out = [os.path.join(INCLUDE, "tets.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PEAKS_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    objdir = os.path.join(ROOT, "_build")
    os.makedirs(objdir, exist_ok=True)
    procs, objs = [], []
    ptmp = PEAKS_LIB + ".tmp"
    procs.append(subprocess.Popen(["nvcc", *ARCH, *FLAGS, "-shared", "-o", ptmp,
                                   os.path.join(CSRC, PEAKS_SOURCE), "-lcudart"]))
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = ["nvcc", *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed")
    tmp = LIB + ".tmp"
    subprocess.check_call(["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    os.replace(ptmp, PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
