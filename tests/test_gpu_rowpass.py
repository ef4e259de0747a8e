"""The row pass (chains along rows out of reach of their neighbours) against the
oracle, bit for bit, and against the general parallel pass on the same inputs.

Lattice starts whose rows lie more than d apart, on cells aligned with the
lattice (one row of disks per cell row), make every chain eligible, so every
claim window runs the row pass (checked through ``row_windows``); a leg longer
than the window of columns a warp holds cancels it, and the general pass must
take over with the same results. With the default cell size some lattice rows
straddle two cell rows; their chains need both, and the general pass runs.
Tolerance: bit-exact (positions, local times, liftings, flags), as for every
parity test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def run(start, ell, n_legs, windows=1, rowpass=True, graph=False, nc=0):
    sysm = ecmc.System(start.x, start.y, start.active, start.box, ell, d=start.d,
                       cells_per_side=nc, log=True, windows=windows, rowpass=rowpass,
                       graph=graph, log_cap=max(1 << 16, 64 * start.k * n_legs * 64))
    flags, done = sysm.run(n_legs)
    assert done == n_legs
    x, y, t, a = sysm.positions()
    log = sysm.liftings()
    st = sysm.stats()
    sysm.close()
    return flags, x, t, a, log, st


def oracle(start, ell, n_legs, windows=1, search=1, nc=0):
    ncell = nc or O.default_cells(start.box, start.d)
    last, legs = O.run_legs(start.x, start.y, start.active, start.box, ell, n_legs,
                            d=start.d, nc=ncell, windows=windows, search=search)
    flags = np.array([r.flag for r in legs], dtype=np.uint8)
    log = np.concatenate([r.log for r in legs])
    last.window_flags = int(sum(int(r.wflags.sum()) for r in legs))
    return flags, last, log


def by_chain(log):
    return log[np.lexsort((np.arange(len(log)), log["c"], log["leg"]))]


def same(g, o):
    gf, gx, gt, ga, glog, st = g
    of, last, olog = o
    assert np.array_equal(gf, of), (gf, of)
    assert np.array_equal(ga, last.active)
    assert np.array_equal(gx, last.x), np.max(np.abs(gx - last.x))
    assert np.array_equal(gt, last.t), np.max(np.abs(gt - last.t))
    a, b = by_chain(olog), by_chain(glog)
    assert len(a) == len(b)
    for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
        assert np.array_equal(a[f], b[f]), f
    assert st["liftings"] == len(olog)
    # the per-window flags: windows whose isolated claim sets met
    assert st["conflict_windows"] == last.window_flags
    assert st["horizon_asserts"] == 0 and st["order_errors"] == 0


@pytest.mark.parametrize("m,eta,k,ell,legs,windows,seed", [
    (32, 0.70, 8, 1.0, 6, 1, 1),      # few chains, few meetings
    (32, 0.70, 64, 1.0, 4, 1, 2),     # dense: components, repairs after the row pass
    (32, 0.70, 200, 1.0, 3, 1, 3),    # most rows hold several chains
    (96, 0.72, 96, 2.0, 3, 1, 4),     # longer legs: wider scans
    (64, 0.708, 64, 1.0, 4, 2, 5),    # claim windows: pauses inside the row pass
    (64, 0.708, 256, 1.0, 3, 5, 6),
    (128, 0.708, 128, 1.0, 3, 1, 7),  # config 2 geometry
])
def test_row_pass_equals_oracle(m, eta, k, ell, legs, windows, seed):
    s = synth.lattice_start(m, eta, k, seed=seed)
    g = run(s, ell, legs, windows, nc=m)
    same(g, oracle(s, ell, legs, windows, nc=m))
    assert g[5]["row_windows"] == legs * windows


@pytest.mark.parametrize("m,k,seed", [(48, 48, 4), (128, 128, 7)])
def test_default_cells_equal_oracle(m, k, seed):
    """Default cell size: whichever pass runs, the oracle's results."""
    s = synth.lattice_start(m, 0.72, k, seed=seed)
    same(run(s, 1.0, 3), oracle(s, 1.0, 3))


@pytest.mark.parametrize("m,k,windows,seed", [(32, 64, 1, 2), (64, 256, 5, 6)])
def test_row_pass_equals_general_pass(m, k, windows, seed):
    """The same inputs through the row pass and through the general pass:
    identical results; only the general pass's own counters differ."""
    s = synth.lattice_start(m, 0.70, k, seed=seed)
    a = run(s, 1.0, 3, windows, rowpass=True, nc=m)
    b = run(s, 1.0, 3, windows, rowpass=False, nc=m)
    assert a[5]["row_windows"] == 3 * windows and b[5]["row_windows"] == 0
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    assert np.array_equal(by_chain(a[4]), by_chain(b[4]))


def test_row_pass_cancelled_by_a_wide_scan():
    """A leg of 8 d: the first scan reaches beyond the warp's columns, the row
    pass cancels itself and the general pass runs the window."""
    s = synth.lattice_start(32, 0.70, 6, seed=11)
    g = run(s, 8.0, 2, nc=32)
    same(g, oracle(s, 8.0, 2, nc=32))
    assert g[5]["row_windows"] < 2


def test_row_pass_not_used_with_rows_in_reach():
    """Staggered rows (pairs of rows closer than d): the general pass."""
    s = synth.staggered_start(40, 0.5, 40, seed=3, row_shift=0.05, pair_shift=0.15)
    g = run(s, 1.0, 2)
    same(g, oracle(s, 1.0, 2))
    assert g[5]["row_windows"] == 0


# ---- the benchmark's settings over many legs (N = 2^20, eta = 0.72)

@pytest.mark.parametrize("k,legs,windows", [(1024, 10, 1), (4096, 3, 1)])
def test_bench_settings_many_legs_cells(k, legs, windows):
    s = synth.lattice_start(1024, 0.72, k, seed=0)
    g = run(s, 1.0, legs, windows, nc=1024)
    same(g, oracle(s, 1.0, legs, windows, nc=1024))
    assert g[5]["row_windows"] == legs * windows


@pytest.mark.parametrize("k,legs", [(1024, 10), (4096, 3)])
def test_bench_settings_many_legs_graph(k, legs):
    s = synth.lattice_start(1024, 0.72, k, seed=0)
    g = run(s, 1.0, legs, graph=True, nc=1024)
    same(g, oracle(s, 1.0, legs, search=2, nc=1024))
