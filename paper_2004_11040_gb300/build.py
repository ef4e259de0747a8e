"""Builds libecmc.so in-tree with nvcc for sm_103a (GB300).

Two translation units -- the cell-scan path with the C ABI (ecmc.cu) and the
constraint-graph path (graph.cu) -- are compiled in parallel, then linked.
"""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
UNITS = [os.path.join(CSRC, "ecmc.cu"), os.path.join(CSRC, "graph.cu")]
HDR = os.path.join(ROOT, "include", "ecmc.h")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libecmc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [
    *ARCH,
    "-lineinfo", "-O3", "-std=c++17",
    "-fmad=false",  # no FMA contraction: FP64 results bit-reproducible
    "-Xcompiler", "-fPIC",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources() -> list[str]:
    return UNITS + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + [HDR, os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(OUT_DIR, os.path.basename(u)[:-3] + tag + ".o") for u in UNITS]
    procs = []
    for u, o in zip(UNITS, objs):
        cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", u, "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
    codes = [p.wait() for p in procs]
    try:
        for u, c in zip(UNITS, codes):
            if c != 0:
                raise subprocess.CalledProcessError(c, f"nvcc {os.path.basename(u)}")
        tmp = LIB + tag
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
