"""ctypes wrapper around ``alg5_openmp.c``: the paper's multithreaded ECMC
(Alg. 5) on the host cores, the multicore CPU baseline of the benchmark.

TEST AND MEASUREMENT INFRASTRUCTURE: only ``tests/`` and ``bench.py``'s CPU
baseline use it. With several chains in flight its result depends on the
thread schedule (a horizon violation is counted, not repaired), so it is a
throughput baseline, not an oracle; with one thread and one chain it equals
the oracle (tested).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from .oracle import default_cells

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alg5_openmp.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libalg5.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC", "-shared",
          "-Wall"]


class A5Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("L", C.c_double), ("d", C.c_double), ("ell", C.c_double),
                ("nc", C.c_int32), ("threads", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile with OpenMP (without it if the compiler has none: one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.a5_run.argtypes = [C.POINTER(A5Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int32, C.c_int32, C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                C.POINTER(C.c_int32)]
        _lib.a5_run.restype = C.c_int
    return _lib


@dataclass
class A5Result:
    x: np.ndarray
    active: np.ndarray
    lifts: int
    violations: int
    seconds: float
    threads: int


def run(x, y, active, L, ell, n_legs, *, d=1.0, nc=None, threads=0) -> A5Result:
    """n_legs legs of Alg. 5 with len(active) chains; inputs are not modified."""
    x = np.array(x, dtype=np.float64, copy=True)
    y = np.ascontiguousarray(y, dtype=np.float64)
    act = np.array(active, dtype=np.int32, copy=True)
    if nc is None:
        nc = default_cells(L, d)
    p = A5Params(x.shape[0], L, d, ell, nc, threads)
    lifts, viol, secs, nth = C.c_int64(0), C.c_int64(0), C.c_double(0.0), C.c_int32(0)
    rc = lib().a5_run(C.byref(p), x.ctypes.data, y.ctypes.data, act.ctypes.data,
                      act.shape[0], n_legs, C.byref(lifts), C.byref(viol), C.byref(secs),
                      C.byref(nth))
    if rc != 0:
        raise RuntimeError(f"a5_run failed: {rc}")
    return A5Result(x=x, active=act, lifts=int(lifts.value), violations=int(viol.value),
                    seconds=float(secs.value), threads=int(nth.value))
