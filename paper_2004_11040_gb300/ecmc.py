"""Python binding of libecmc (include/ecmc.h): argument marshalling only.

Every step of the ECMC path runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers and C return codes to exceptions.
If the shared library is missing the import fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ECMC_OK = 0
ECMC_EINVAL = -1
ECMC_ENOMEM = -2
ECMC_ECUDA = -3
ECMC_ETIMEOUT = -4
ECMC_ECAPACITY = -5
ECMC_LOG_LIFTINGS = 0x1
ECMC_INPUT_DEVICE = 0x2
ECMC_GRAPH = 0x4
ECMC_RESTART = 0x8
ECMC_NO_ROWPASS = 0x10

EXPORTS = ("ecmc_create", "ecmc_run_to_breakpoint", "ecmc_positions", "ecmc_stats",
           "ecmc_profile", "ecmc_liftings", "ecmc_destroy", "ecmc_last_error",
           "ecmc_batch_create", "ecmc_batch_run", "ecmc_batch_last_error",
           "ecmc_batch_destroy", "ecmc_leg_noalloc", "ecmc_set_direction",
           "ecmc_graph_arrows", "ecmc_set_wait_limit", "ecmc_context_bytes",
           "ecmc_set_cache_limit", "ecmc_cache_info")


class ecmc_params(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double), ("d", C.c_double), ("ell", C.c_double),
                ("n_chains", C.c_int32), ("cells_per_side", C.c_int32), ("flags", C.c_uint32),
                ("undo_cap", C.c_int32), ("log_cap", C.c_int64), ("windows", C.c_int32),
                ("reserved", C.c_int32)]


class ecmc_stats_t(C.Structure):
    _fields_ = [("liftings", C.c_int64), ("legs", C.c_int64), ("conflict_legs", C.c_int64),
                ("repaired_chains", C.c_int64), ("horizon_asserts", C.c_int64),
                ("order_errors", C.c_int64), ("device_ms", C.c_double),
                ("continued_chains", C.c_int64), ("restarts", C.c_int64),
                ("row_windows", C.c_int64), ("device_bytes", C.c_int64),
                ("blocked_chains", C.c_int64), ("conflict_windows", C.c_int64)]


class ecmc_profile_t(C.Structure):
    _fields_ = [("pass1_launches", C.c_int64), ("repair_launches", C.c_int64),
                ("other_launches", C.c_int64), ("pass1_liftings", C.c_int64),
                ("repair_liftings", C.c_int64), ("pass1_ms", C.c_double),
                ("repair_ms", C.c_double), ("other_ms", C.c_double)]


LIFT_DTYPE = np.dtype([("leg", np.int32), ("c", np.int32), ("i", np.int32), ("j", np.int32),
                       ("t", np.float64), ("tau", np.float64), ("xi", np.float64),
                       ("xj", np.float64)])


class EcmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libecmc error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    """Path of the in-tree libecmc.so."""
    return _build.LIB


def load(path: str | None = None):
    """Loads libecmc.so (built in-tree by build.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libecmc not built: {path} missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.ecmc_create.argtypes = [C.POINTER(ecmc_params), vp, vp, vp, vp, C.POINTER(vp)]
    lib.ecmc_create.restype = C.c_int
    lib.ecmc_run_to_breakpoint.argtypes = [vp, C.c_int32, C.c_uint64, vp, C.POINTER(C.c_int32)]
    lib.ecmc_run_to_breakpoint.restype = C.c_int
    lib.ecmc_positions.argtypes = [vp, vp, vp, vp, vp]
    lib.ecmc_positions.restype = C.c_int
    lib.ecmc_set_direction.argtypes = [vp, C.c_int32]
    lib.ecmc_set_direction.restype = C.c_int
    lib.ecmc_set_wait_limit.argtypes = [vp, C.c_uint64]
    lib.ecmc_set_wait_limit.restype = C.c_int
    lib.ecmc_context_bytes.argtypes = [C.POINTER(ecmc_params), C.POINTER(C.c_int64)]
    lib.ecmc_context_bytes.restype = C.c_int
    lib.ecmc_set_cache_limit.argtypes = [C.c_int64]
    lib.ecmc_set_cache_limit.restype = C.c_int
    lib.ecmc_cache_info.argtypes = [C.POINTER(C.c_int64)] * 4
    lib.ecmc_cache_info.restype = C.c_int
    lib.ecmc_stats.argtypes = [vp, C.POINTER(ecmc_stats_t)]
    lib.ecmc_stats.restype = C.c_int
    lib.ecmc_profile.argtypes = [vp, C.POINTER(ecmc_profile_t)]
    lib.ecmc_profile.restype = C.c_int
    lib.ecmc_graph_arrows.argtypes = [vp, vp, vp]
    lib.ecmc_graph_arrows.restype = C.c_int
    lib.ecmc_liftings.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
    lib.ecmc_liftings.restype = C.c_int
    lib.ecmc_destroy.argtypes = [vp]
    lib.ecmc_destroy.restype = None
    lib.ecmc_last_error.argtypes = [vp]
    lib.ecmc_last_error.restype = C.c_char_p
    lib.ecmc_batch_create.argtypes = [vp, C.POINTER(vp)]
    lib.ecmc_batch_create.restype = C.c_int
    lib.ecmc_batch_run.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp, vp,
                                   C.POINTER(C.c_double)]
    lib.ecmc_batch_run.restype = C.c_int
    lib.ecmc_batch_last_error.argtypes = [vp]
    lib.ecmc_batch_last_error.restype = C.c_char_p
    lib.ecmc_batch_destroy.argtypes = [vp]
    lib.ecmc_batch_destroy.restype = None
    lib.ecmc_leg_noalloc.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int32,
                                     C.c_int32, vp, vp, vp, vp, vp, C.POINTER(C.c_uint8),
                                     C.POINTER(C.c_int64)]
    lib.ecmc_leg_noalloc.restype = C.c_int
    _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != ECMC_OK:
        msg = load().ecmc_last_error(ctx)
        raise EcmcError(rc, (msg or b"").decode())


def _ptr(a):
    """Data pointer of a C-contiguous numpy array or torch tensor (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags.c_contiguous
    return a.ctypes.data


def ecmc_create(params: ecmc_params, x, y, active, stream=None):
    """Context for a lifted configuration; x, y, active as numpy (host) or,
    with ECMC_INPUT_DEVICE in params.flags, CUDA tensors."""
    lib = load()
    out = C.c_void_p()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    _check(lib.ecmc_create(C.byref(params), _ptr(x), _ptr(y), _ptr(active), st, C.byref(out)))
    return out


def ecmc_run_to_breakpoint(ctx, n_legs: int, event_budget: int = 0, leg_flags_out=None):
    """Runs legs; returns legs done. leg_flags_out: uint8 array of n_legs or None."""
    done = C.c_int32()
    _check(load().ecmc_run_to_breakpoint(ctx, n_legs, event_budget, _ptr(leg_flags_out),
                                         C.byref(done)), ctx)
    return done.value


def ecmc_positions(ctx, x=None, y=None, t=None, active=None):
    _check(load().ecmc_positions(ctx, _ptr(x), _ptr(y), _ptr(t), _ptr(active)), ctx)


def ecmc_context_bytes(params) -> int:
    """Device bytes a context created with `params` would hold (nothing allocated)."""
    out = C.c_int64()
    rc = load().ecmc_context_bytes(C.byref(params), C.byref(out))
    if rc != ECMC_OK:
        raise EcmcError(rc, "ecmc_context_bytes")
    return int(out.value)


def ecmc_set_cache_limit(nbytes: int):
    """Bound on the device bytes the library keeps for reuse per device (0: none)."""
    _check(load().ecmc_set_cache_limit(int(nbytes)))


def ecmc_cache_info() -> dict:
    """The device memory cache: bytes cached and in use, hits and misses."""
    v = [C.c_int64() for _ in range(4)]
    _check(load().ecmc_cache_info(*[C.byref(x) for x in v]))
    return dict(zip(("cached_bytes", "in_use_bytes", "hits", "misses"), (x.value for x in v)))


def ecmc_set_wait_limit(ctx, ns: int):
    """Bound (ns) on every device wait of the context's persistent kernels."""
    _check(load().ecmc_set_wait_limit(ctx, int(ns)), ctx)


def ecmc_set_direction(ctx, direction: int):
    """0: legs move +x (after creation); 1: legs move +y."""
    _check(load().ecmc_set_direction(ctx, int(direction)), ctx)


def ecmc_stats(ctx) -> dict:
    st = ecmc_stats_t()
    _check(load().ecmc_stats(ctx, C.byref(st)), ctx)
    return {f: getattr(st, f) for f, _ in ecmc_stats_t._fields_}


def ecmc_profile(ctx) -> dict:
    pr = ecmc_profile_t()
    _check(load().ecmc_profile(ctx, C.byref(pr)), ctx)
    return {f: getattr(pr, f) for f, _ in ecmc_profile_t._fields_}


def ecmc_liftings(ctx) -> np.ndarray:
    n = C.c_int64()
    _check(load().ecmc_liftings(ctx, None, 0, C.byref(n)), ctx)
    buf = np.zeros(n.value, dtype=LIFT_DTYPE)
    _check(load().ecmc_liftings(ctx, _ptr(buf) if n.value else None, n.value, C.byref(n)), ctx)
    return buf


def ecmc_graph_arrows(ctx, n: int):
    """Arrows of G(3) and their b_ij, int32 and float64 arrays [n, 3] (-1 and
    0 where a corridor is empty), in the context's current frame."""
    a = np.empty((n, 3), dtype=np.int32)
    b = np.empty((n, 3), dtype=np.float64)
    _check(load().ecmc_graph_arrows(ctx, _ptr(a), _ptr(b)), ctx)
    return a, b


def ecmc_leg_noalloc(n, box, d, ell, n_chains, cells_per_side, x, y, active, t_out=None,
                     stream=None):
    """One leg through the entry point that allocates nothing (device tensors
    in and out); returns (flag, liftings). Raises EcmcError on a failure code."""
    flag = C.c_uint8()
    lifts = C.c_int64()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    rc = load().ecmc_leg_noalloc(int(n), float(box), float(d), float(ell), int(n_chains),
                                 int(cells_per_side), _ptr(x), _ptr(y), _ptr(active),
                                 _ptr(t_out), st, C.byref(flag), C.byref(lifts))
    if rc != ECMC_OK:
        raise EcmcError(rc, "ecmc_leg_noalloc failed")
    return flag.value, lifts.value


def ecmc_destroy(ctx):
    load().ecmc_destroy(ctx)


def ecmc_last_error(ctx=None) -> str:
    return (load().ecmc_last_error(ctx) or b"").decode()


def ecmc_batch_create(stream=None):
    out = C.c_void_p()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    rc = load().ecmc_batch_create(st, C.byref(out))
    if rc != ECMC_OK:
        raise EcmcError(rc, "ecmc_batch_create failed")
    return out


def ecmc_batch_run(batch, ctxs, max_legs, budgets=None):
    """One persistent launch over the contexts; returns (liftings, legs, ms)."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    bud = None
    if budgets is not None:
        bud = np.ascontiguousarray(budgets, dtype=np.uint64)
    lifts = np.zeros(n, dtype=np.int64)
    legs = np.zeros(n, dtype=np.int32)
    ms = C.c_double()
    rc = load().ecmc_batch_run(batch, C.cast(arr, C.c_void_p), n, int(max_legs),
                               _ptr(bud) if bud is not None else None, _ptr(lifts), _ptr(legs),
                               C.byref(ms))
    if rc != ECMC_OK:
        msg = (load().ecmc_batch_last_error(batch) or b"").decode()
        raise EcmcError(rc, msg)
    return lifts, legs, ms.value


def ecmc_batch_destroy(batch):
    load().ecmc_batch_destroy(batch)


class System:
    """One ECMC system on the GPU: a thin owner of an ecmc_ctx handle."""

    def __init__(self, x, y, active, box, ell, *, d=1.0, cells_per_side=0, log=False,
                 undo_cap=0, log_cap=0, stream=None, device_input=False, windows=1,
                 graph=False, restart=False, rowpass=True):
        x = x if device_input else np.ascontiguousarray(x, dtype=np.float64)
        y = y if device_input else np.ascontiguousarray(y, dtype=np.float64)
        active = active if device_input else np.ascontiguousarray(active, dtype=np.int32)
        self.n = int(x.shape[0])
        self.k = int(active.shape[0])
        flags = (ECMC_LOG_LIFTINGS if log else 0) | (ECMC_INPUT_DEVICE if device_input else 0) \
            | (ECMC_GRAPH if graph else 0) | (ECMC_RESTART if restart else 0) \
            | (0 if rowpass else ECMC_NO_ROWPASS)
        self.params = ecmc_params(self.n, float(box), float(d), float(ell), self.k,
                                  int(cells_per_side), flags, int(undo_cap), int(log_cap),
                                  int(windows), 0)
        self.ctx = ecmc_create(self.params, x, y, active, stream)

    def run(self, n_legs, event_budget=0):
        flags = np.zeros(max(n_legs, 1), dtype=np.uint8)
        done = ecmc_run_to_breakpoint(self.ctx, n_legs, event_budget, flags)
        return flags[:done], done

    def positions(self):
        x = np.empty(self.n)
        y = np.empty(self.n)
        t = np.empty(self.n)
        a = np.empty(self.k, dtype=np.int32)
        ecmc_positions(self.ctx, x, y, t, a)
        return x, y, t, a

    def stats(self):
        return ecmc_stats(self.ctx)

    def set_wait_limit(self, ns: int):
        ecmc_set_wait_limit(self.ctx, ns)

    def set_direction(self, direction: int):
        ecmc_set_direction(self.ctx, direction)

    def liftings(self):
        return ecmc_liftings(self.ctx)

    def arrows(self):
        return ecmc_graph_arrows(self.ctx, self.n)

    def profile(self):
        return ecmc_profile(self.ctx)

    def close(self):
        if self.ctx:
            ecmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
