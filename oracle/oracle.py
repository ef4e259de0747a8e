"""ctypes wrapper around the plain C oracle (``ecmc_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use this module. The product path (the CUDA library)
never imports or links it.

The oracle computes Alg. 2 of the paper (ECMC with global time) between two
breakpoints, the leg's conflict flag from isolated chain runs, Alg. 4 for the
Lemma 2 self-check, and the constraint graph G(3) of Sec. 3.1; see the header
of ``ecmc_oracle.c`` for the readings. ``search`` selects how a step finds its
candidates: 0 every pair (the definition), 1 the cell scan, 2 the arrows of
G(3); the events are those of Alg. 2 in every case, the flag depends on it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ecmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
          "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE doubles)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class LiftRec(C.Structure):
    _fields_ = [("leg", C.c_int32), ("c", C.c_int32), ("i", C.c_int32), ("j", C.c_int32),
                ("t", C.c_double), ("tau", C.c_double), ("xi", C.c_double), ("xj", C.c_double)]


LIFT_DTYPE = np.dtype([("leg", np.int32), ("c", np.int32), ("i", np.int32), ("j", np.int32),
                       ("t", np.float64), ("tau", np.float64), ("xi", np.float64),
                       ("xj", np.float64)])


class Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("L", C.c_double), ("d", C.c_double), ("ell", C.c_double),
                ("nc", C.c_int32), ("search", C.c_int32), ("windows", C.c_int32),
                ("pad", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        _lib.orc_leg.argtypes = [C.POINTER(Params), C.c_int32, dp, dp, dp, C.c_int32, ip,
                                 C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_uint8), C.POINTER(C.c_int64), C.c_void_p,
                                 C.c_void_p]
        _lib.orc_leg.restype = C.c_int
        _lib.orc_alg4_leg.argtypes = [C.POINTER(Params), C.c_int32, dp, dp, dp, C.c_int32, ip,
                                      C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
        _lib.orc_alg4_leg.restype = C.c_int
        _lib.orc_step.argtypes = [C.POINTER(Params), dp, dp, C.c_void_p, C.c_void_p, C.c_int32,
                                  C.c_double, ip, ip, dp, ip]
        _lib.orc_step.restype = C.c_int
        _lib.orc_claim_set.argtypes = [C.POINTER(Params), dp, dp, C.c_int32, ip, C.c_int64,
                                       C.POINTER(C.c_int64)]
        _lib.orc_claim_set.restype = C.c_int
        _lib.orc_graph3.argtypes = [C.POINTER(Params), dp, dp, C.c_int32, C.c_void_p, C.c_int64,
                                    ip]
        _lib.orc_graph3.restype = C.c_int
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def default_cells(L: float, d: float = 1.0) -> int:
    """Largest nc with cell side a = L/nc >= d*(1 + 2^-20) (and nc >= 3)."""
    nc = int(L / (d * (1.0 + 2.0 ** -20)))
    while nc > 3 and not (L / nc >= d * (1.0 + 2.0 ** -20)):
        nc -= 1
    if nc < 3:
        raise ValueError("box too small: need L >= 3 cells of side > d")
    return nc


@dataclass
class LegResult:
    x: np.ndarray
    t: np.ndarray
    active: np.ndarray
    flag: int
    lifts: int
    lifts_per_chain: np.ndarray
    log: np.ndarray = field(default_factory=lambda: np.zeros(0, LIFT_DTYPE))
    wflags: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))


class OracleError(RuntimeError):
    pass


def run_leg(x, y, active, L, ell, *, d=1.0, nc=None, search=1, leg=0, log=True,
            log_cap=None, windows=1) -> LegResult:
    """One leg of Alg. 2 (global time) with the conflict flag. Inputs are not modified."""
    x = np.array(x, dtype=np.float64, copy=True)
    y = np.ascontiguousarray(y, dtype=np.float64)
    act = np.array(active, dtype=np.int32, copy=True)
    n, k = x.shape[0], act.shape[0]
    if nc is None:
        nc = default_cells(L, d)
    p = Params(n, L, d, ell, nc, search, windows, 0)
    t = np.zeros(n, dtype=np.float64)
    if log_cap is None:
        log_cap = max(1024, int(64 * k * (ell + 1.0) / 0.01) if log else 0)
        log_cap = min(log_cap, 50_000_000)
    logbuf = np.zeros(log_cap if log else 0, dtype=LIFT_DTYPE)
    log_n = C.c_int64(0)
    flag = C.c_uint8(0)
    lifts = C.c_int64(0)
    per_chain = np.zeros(k, dtype=np.int64)
    wflags = np.zeros(max(1, windows), dtype=np.uint8)
    rc = lib().orc_leg(C.byref(p), leg, _dptr(x), _dptr(y), _dptr(t), k, _iptr(act),
                       logbuf.ctypes.data if log else None, log_cap, C.byref(log_n),
                       C.byref(flag), C.byref(lifts), per_chain.ctypes.data,
                       wflags.ctypes.data)
    if rc != 0:
        raise OracleError(f"orc_leg failed: {rc}")
    return LegResult(x=x, t=t, active=act, flag=int(flag.value), lifts=int(lifts.value),
                     lifts_per_chain=per_chain, log=logbuf[: log_n.value].copy(),
                     wflags=wflags)


def run_legs(x, y, active, L, ell, n_legs, **kw) -> tuple[LegResult, list[LegResult]]:
    """n_legs consecutive legs; chains continue from their stalled disks."""
    legs = []
    cur_x, cur_a = np.array(x, dtype=np.float64), np.array(active, dtype=np.int32)
    for leg in range(n_legs):
        r = run_leg(cur_x, y, cur_a, L, ell, leg=leg, **kw)
        legs.append(r)
        cur_x, cur_a = r.x, r.active
    return legs[-1], legs


def run_alg4_leg(x, y, active, L, ell, *, d=1.0, leg=0):
    """Alg. 4 over one leg; returns (status, x, t, active, log). status 0 = ok."""
    x = np.array(x, dtype=np.float64, copy=True)
    y = np.ascontiguousarray(y, dtype=np.float64)
    act = np.array(active, dtype=np.int32, copy=True)
    n, k = x.shape[0], act.shape[0]
    p = Params(n, L, d, ell, 3, 0, 1, 0)
    t = np.zeros(n, dtype=np.float64)
    cap = 1_000_000
    logbuf = np.zeros(cap, dtype=LIFT_DTYPE)
    log_n = C.c_int64(0)
    rc = lib().orc_alg4_leg(C.byref(p), leg, _dptr(x), _dptr(y), _dptr(t), k, _iptr(act),
                            logbuf.ctypes.data, cap, C.byref(log_n))
    return rc, x, t, act, logbuf[: log_n.value].copy()


def step(x, y, i, D, L, *, d=1.0, nc=None, search=0, tag=None, t=None):
    """Single step of a chain: (lift, j, tau, mlast)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if nc is None:
        nc = default_cells(L, d)
    p = Params(x.shape[0], L, d, 0.0, nc, search, 1, 0)
    lift, j, m = C.c_int32(), C.c_int32(), C.c_int32()
    tau = C.c_double()
    tg = None
    if tag is not None:
        tg = np.ascontiguousarray(tag, dtype=np.int8)
    tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
    rc = lib().orc_step(C.byref(p), _dptr(x), _dptr(y), tt.ctypes.data if tt is not None else None,
                        tg.ctypes.data if tg is not None else None,
                        i, D, C.byref(lift), C.byref(j), C.byref(tau), C.byref(m))
    if rc != 0:
        raise OracleError(f"orc_step failed: {rc}")
    return lift.value, j.value, tau.value, m.value


def claim_set(x, y, i0, L, ell, *, d=1.0, nc=None) -> np.ndarray:
    """Cells scanned by chain starting at i0 when run alone for one leg."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if nc is None:
        nc = default_cells(L, d)
    p = Params(x.shape[0], L, d, ell, nc, 1, 1, 0)
    cap = nc * nc
    cells = np.zeros(cap, dtype=np.int32)
    n_out = C.c_int64()
    rc = lib().orc_claim_set(C.byref(p), _dptr(x), _dptr(y), i0, _iptr(cells), cap,
                             C.byref(n_out))
    if rc != 0:
        raise OracleError(f"orc_claim_set failed: {rc}")
    return cells[: n_out.value].copy()


def graph3(x, y, L, *, d=1.0, nc=None, search=0, ids=None) -> np.ndarray:
    """Arrows of G(3) (Sec. 3.1): an int32 array [m, 3] (corridor 0 centre,
    1 upper, 2 lower; -1 = empty corridor) for the disks ``ids`` (all disks by
    default). search 0: every pair (the definition); 1: the cell scan."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if nc is None:
        nc = default_cells(L, d)
    p = Params(x.shape[0], L, d, 0.0, nc, 1, 1, 0)
    if ids is None:
        m = x.shape[0]
        idp = None
    else:
        ida = np.ascontiguousarray(ids, dtype=np.int32)
        m = ida.shape[0]
        idp = ida.ctypes.data
    out = np.zeros((m, 3), dtype=np.int32)
    rc = lib().orc_graph3(C.byref(p), _dptr(x), _dptr(y), search, idp, m, _iptr(out))
    if rc != 0:
        raise OracleError(f"orc_graph3 failed: {rc}")
    return out
