"""Constraint-graph mode (ECMC_GRAPH, Sec. 3.1) of libecmc against the oracle.

The oracle's graph-mode legs (search=2) take the liftings of Alg. 2 (pinned
equal to the all-pairs definition in test_oracle_graph.py) and the flag from
the disks isolated chains read. Tolerance: bit-exact, as for the cell scan.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def chain_order(log):
    idx = np.lexsort((np.arange(len(log)), log["c"], log["leg"]))
    return log[idx]


def gpu_graph(start, ell, n_legs, windows=1, undo_cap=0, directions=None):
    sysm = ecmc.System(start.x, start.y, start.active, start.box, ell, d=start.d, log=True,
                       undo_cap=undo_cap, log_cap=max(1 << 16, 64 * start.k * n_legs * 64),
                       windows=windows, graph=True)
    flags = []
    if directions is None:
        f, done = sysm.run(n_legs)
        assert done == n_legs
        flags = list(f)
    else:
        for leg in range(n_legs):
            sysm.set_direction(directions[leg])
            f, done = sysm.run(1)
            assert done == 1
            flags += list(f)
    x, y, t, a = sysm.positions()
    log = sysm.liftings()
    st = sysm.stats()
    sysm.close()
    return np.array(flags, dtype=np.uint8), x, y, t, a, log, st


def oracle_graph(start, ell, n_legs, windows=1):
    last, legs = O.run_legs(start.x, start.y, start.active, start.box, ell, n_legs,
                            d=start.d, windows=windows, search=2)
    flags = np.array([r.flag for r in legs], dtype=np.uint8)
    log = np.concatenate([r.log for r in legs])
    last.window_flags = int(sum(int(r.wflags.sum()) for r in legs))
    return flags, last, log


def assert_graph_parity(start, ell, n_legs, windows=1):
    gf, gx, gy, gt, ga, glog, st = gpu_graph(start, ell, n_legs, windows)
    of, last, olog = oracle_graph(start, ell, n_legs, windows)
    assert np.array_equal(gy, start.y)
    assert np.array_equal(gf, of), (gf, of)
    assert np.array_equal(ga, last.active)
    assert np.array_equal(gx, last.x), np.max(np.abs(gx - last.x))
    assert np.array_equal(gt, last.t), np.max(np.abs(gt - last.t))
    a, b = chain_order(olog), chain_order(glog)
    assert len(a) == len(b)
    for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
        assert np.array_equal(a[f], b[f]), f
    assert st["liftings"] == len(olog)
    assert st["conflict_windows"] == last.window_flags
    assert st["horizon_asserts"] == 0
    assert st["order_errors"] == 0
    return gf, st


@pytest.mark.parametrize("seed", range(6))
def test_graph_config1_lattice_n256(seed):
    s = synth.lattice_start(16, 0.70, 4, seed=seed)
    assert_graph_parity(s, 0.5, 8)


@pytest.mark.parametrize("seed,windows", [(21, 1), (22, 3), (23, 2)])
def test_graph_random_2d(seed, windows):
    """Random (RSA) starts: all three corridors in use, cross-row liftings."""
    s = synth.rsa_start(400, 0.5, 16, seed=seed)
    flags, st = assert_graph_parity(s, 1.5, 6, windows)
    assert st["liftings"] > 500


def test_graph_dense_chains_large_components():
    """Many chains on a small lattice: conflict components of more than 32
    chains replayed in global order."""
    s = synth.lattice_start(16, 0.70, 120, seed=5)
    flags, st = assert_graph_parity(s, 1.0, 4)
    assert flags.all()
    assert st["repaired_chains"] > 0


def test_graph_config2_lattice_n16384():
    s = synth.lattice_start(128, 0.708, 128, seed=7)
    flags, st = assert_graph_parity(s, 1.0, 3)
    assert st["liftings"] > 5000


def test_graph_config3_lattice_n1m_one_leg():
    """N=2^20 (1024x1024), eta=0.72, 1024 chains, ell=1, two claim windows."""
    s = synth.lattice_start(1024, 0.72, 1024, seed=3)
    assert_graph_parity(s, 1.0, 1, windows=2)


def test_graph_equals_cell_scan_results():
    """Both modes compute Alg. 2: positions and liftings agree; only the flags
    (cells vs disks) may differ."""
    s = synth.rsa_start(300, 0.45, 12, seed=31)
    gf, gx, _, gt, ga, glog, _ = gpu_graph(s, 1.2, 5)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.2, log=True)
    sysm.run(5)
    x, _, t, a = sysm.positions()
    clog = sysm.liftings()
    sysm.close()
    assert np.array_equal(gx, x) and np.array_equal(gt, t) and np.array_equal(ga, a)
    a1, b1 = chain_order(glog), chain_order(clog)
    for f in ("leg", "c", "i", "j", "t"):
        assert np.array_equal(a1[f], b1[f]), f


@pytest.mark.parametrize("kind", ["lattice", "rsa"])
def test_graph_direction_alternation(kind):
    """+x / +y legs: the graph is rebuilt for every direction; a +y leg equals
    the oracle's +x leg on exchanged coordinates."""
    if kind == "lattice":
        s = synth.lattice_start(16, 0.70, 6, seed=2)
    else:
        s = synth.rsa_start(300, 0.45, 8, seed=3)
    n_legs = 6
    dirs = [leg % 2 for leg in range(n_legs)]
    gf, gx, gy, gt, ga, glog, st = gpu_graph(s, 0.8, n_legs, directions=dirs)
    x, y, act = s.x.copy(), s.y.copy(), s.active.copy()
    oflags = []
    for leg in range(n_legs):
        if dirs[leg] == 0:
            r = O.run_leg(x, y, act, s.box, 0.8, search=2)
            x = r.x
        else:
            r = O.run_leg(y, x, act, s.box, 0.8, search=2)
            y = r.x
        act = r.active
        oflags.append(r.flag)
    assert np.array_equal(gx, x) and np.array_equal(gy, y)
    assert np.array_equal(ga, act)
    assert np.array_equal(gf, np.array(oflags, dtype=np.uint8))
    assert st["horizon_asserts"] == 0 and st["order_errors"] == 0


def test_graph_event_budget_stops_at_a_breakpoint():
    """An event budget ends the run at the first breakpoint where the liftings
    of the call reach it; the state is that of the oracle after as many legs."""
    s = synth.lattice_start(16, 0.70, 6, seed=4)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 0.6, graph=True)
    flags, done = sysm.run(20, event_budget=60)
    x, y, t, a = sysm.positions()
    st = sysm.stats()
    sysm.close()
    assert 1 <= done < 20
    last, legs = O.run_legs(s.x, s.y, s.active, s.box, 0.6, done, search=2)
    lifts = [r.lifts for r in legs]
    assert sum(lifts) >= 60 and sum(lifts[:-1]) < 60
    assert st["liftings"] == sum(lifts)
    assert np.array_equal(flags, np.array([r.flag for r in legs], dtype=np.uint8))
    assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
    assert np.array_equal(a, last.active)


def test_graph_split_runs_equal_one_run():
    """Legs are independent of how calls cut them: 2 + 4 legs equal 6 legs,
    lifting log (leg indices included) and flags alike."""
    s = synth.rsa_start(250, 0.45, 10, seed=17)
    out = []
    for cuts in ([6], [2, 4], [1, 1, 4]):
        sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, log=True, graph=True)
        flags = []
        for n in cuts:
            f, done = sysm.run(n)
            assert done == n
            flags += list(f)
        x, y, t, a = sysm.positions()
        log = chain_order(sysm.liftings())
        sysm.close()
        out.append((x, t, a, np.array(flags), log))
    for o in out[1:]:
        for u, v in zip(out[0][:4], o[:4]):
            assert np.array_equal(u, v)
        for f in ("leg", "c", "i", "j", "t"):
            assert np.array_equal(out[0][4][f], o[4][f]), f


def _restart_run(s, ell, n_legs):
    sysm = ecmc.System(s.x, s.y, s.active, s.box, ell, log=True, graph=True, restart=True,
                       log_cap=max(1 << 16, 64 * s.k * n_legs * 64))
    flags, done = sysm.run(n_legs)
    assert done == n_legs
    x, y, t, a = sysm.positions()
    log = chain_order(sysm.liftings())
    st = sysm.stats()
    sysm.close()
    return flags, x, t, a, log, st


@pytest.mark.parametrize("kind,seed", [("lattice", 1), ("lattice", 2), ("rsa", 3), ("rsa", 4)])
def test_restart_mode_equals_oracle(kind, seed):
    """Restart strategy 2 (Sec. 3.4): passes cut at the earliest stop time T*
    and begun again from it give the oracle's legs exactly; the leg flag is
    that of the first pass, the oracle's one-window flag."""
    if kind == "lattice":
        s = synth.lattice_start(24, 0.70, 12, seed=seed)
        ell, n_legs = 1.0, 6
    else:
        s = synth.rsa_start(400, 0.5, 16, seed=seed)
        ell, n_legs = 1.5, 5
    flags, x, t, a, log, st = _restart_run(s, ell, n_legs)
    of, last, olog = oracle_graph(s, ell, n_legs)
    assert np.array_equal(flags, of)
    assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
    assert np.array_equal(a, last.active)
    o = chain_order(olog)
    for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
        assert np.array_equal(o[f], log[f]), f
    assert st["conflict_windows"] == last.window_flags == int(of.sum())
    assert st["horizon_asserts"] == 0 and st["order_errors"] == 0


def test_restart_mode_two_chains_in_a_row():
    """The rear chain of one lattice row reaches the front chain's start disk
    after a few liftings: the first pass stops there at T* > 0, both chains
    go back to T*, and the leg goes on from T* as from a breakpoint."""
    m, r = 16, 5
    s = synth.lattice_start(m, 0.70, 2, seed=3)
    s.active = np.array([0 * m + r, 5 * m + r], dtype=np.int32)  # columns 0 and 5 of row r
    flags, x, t, a, log, st = _restart_run(s, 0.5, 3)
    of, last, olog = oracle_graph(s, 0.5, 3)
    assert np.array_equal(flags, of) and flags[0] == 1
    assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
    assert np.array_equal(a, last.active)
    o = chain_order(olog)
    for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
        assert np.array_equal(o[f], log[f]), f
    assert st["restarts"] >= 1


def test_restart_mode_n1m():
    """N = 2^20, k = 1024: one leg against the oracle (passes that cannot
    progress fall back to the local repair)."""
    s = synth.lattice_start(1024, 0.72, 1024, seed=5)
    flags, x, t, a, log, st = _restart_run(s, 1.0, 1)
    of, last, olog = oracle_graph(s, 1.0, 1)
    assert np.array_equal(flags, of)
    assert np.array_equal(x, last.x) and np.array_equal(a, last.active)


def test_restart_needs_graph_and_one_window():
    s = synth.lattice_start(16, 0.70, 4, seed=0)
    for kw in ({"graph": False}, {"graph": True, "windows": 2}):
        with pytest.raises(ecmc.EcmcError) as e:
            ecmc.System(s.x, s.y, s.active, s.box, 0.5, restart=True, **kw)
        assert e.value.code == ecmc.ECMC_EINVAL


def _b_of(x, y, a, L, d):
    """b_ij = sqrt(d^2 - dy^2) of each arrow (dy minimum image), 0 for none."""
    i = np.repeat(np.arange(len(x)), 3).reshape(-1, 3)
    j = np.where(a >= 0, a, 0)
    ay = np.abs(y[j] - y[i])
    la = L - ay
    ay = np.where(la < ay, la, ay)
    return np.where(a >= 0, np.sqrt(d * d - ay * ay), 0.0)


@pytest.mark.parametrize("kind,search", [("lattice16", 0), ("rsa", 0), ("rsa_dense", 0),
                                         ("lattice128", 1), ("lattice1024", 1)])
def test_graph_arrows_equal_oracle(kind, search):
    """The arrows the device builds equal the oracle's G(3), all pairs (the
    definition) on small starts and its cell scan on large ones, and every b_ij
    is sqrt(d^2 - dy^2) of its arrow, bit for bit."""
    if kind == "lattice16":
        s = synth.lattice_start(16, 0.70, 4, seed=1)
    elif kind == "rsa":
        s = synth.rsa_start(500, 0.5, 8, seed=41)
    elif kind == "rsa_dense":
        s = synth.rsa_start(600, 0.52, 8, seed=42)
    elif kind == "lattice128":
        s = synth.lattice_start(128, 0.708, 128, seed=7)
    else:
        s = synth.lattice_start(1024, 0.72, 1024, seed=3)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d, graph=True)
    a, b = sysm.arrows()
    sysm.close()
    ids = np.arange(s.n)
    if s.n > 100_000:  # the oracle's build takes seconds per 10^5 disks: a sample
        rng = np.random.default_rng(5)
        ids = np.unique(np.concatenate([np.arange(2048), s.n - 1 - np.arange(2048),
                                        rng.choice(s.n, 16384, replace=False)]))
    ref = O.graph3(s.x, s.y, s.box, d=s.d, search=search, ids=ids)
    assert np.array_equal(a[ids], ref)
    assert np.array_equal(b, _b_of(s.x, s.y, a, s.box, s.d))
    if kind.startswith("rsa"):
        assert (a[:, 1:] >= 0).any()  # the side corridors are in use


def test_graph_arrows_after_direction_change():
    """After set_direction(1) the graph is that of +x motion in the exchanged
    frame: G(3) of (y, x)."""
    s = synth.rsa_start(400, 0.5, 8, seed=43)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, d=s.d, graph=True)
    sysm.set_direction(1)
    a, b = sysm.arrows()
    sysm.close()
    ref = O.graph3(s.y, s.x, s.box, d=s.d, search=0)
    assert np.array_equal(a, ref)
    assert np.array_equal(b, _b_of(s.y, s.x, ref, s.box, s.d))


def test_graph_arrows_need_a_graph_context():
    s = synth.lattice_start(16, 0.70, 4, seed=0)
    sysm = ecmc.System(s.x, s.y, s.active, s.box, 0.5)
    with pytest.raises(ecmc.EcmcError) as e:
        sysm.arrows()
    sysm.close()
    assert e.value.code == ecmc.ECMC_EINVAL


def test_graph_inputs_checked():
    """Out-of-box coordinates and repeated or out-of-range active ids are
    reported as EINVAL by the device-side check, before the graph is built."""
    s = synth.lattice_start(8, 0.6, 2, seed=1)
    for x, act in ((s.x, [0, 0]), (s.x, [0, s.n]), (np.where(np.arange(s.n) == 3, s.box, s.x),
                                                     [0, 1])):
        with pytest.raises(ecmc.EcmcError) as e:
            ecmc.System(x, s.y, act, s.box, 1.0, graph=True)
        assert e.value.code == ecmc.ECMC_EINVAL
