"""Pins for the CPU oracle against facts the paper and the mathematics fix.

Each test names the passage it follows. None of these compares the oracle with
itself: the expected values are closed forms, invariants stated in the paper,
exact-rational brute force, or an independent formulation (Alg. 4).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import synth


def ulp(v):
    return np.spacing(abs(v))


# ---------------------------------------------------------------- synth


def test_splitmix64_published_vector():
    # Reference outputs of SplitMix64 for seed 1234567 (Steele, Lea & Flood 2014;
    # the common splitmix64.c next() sequence).
    v = synth.splitmix64(1234567, 0, 3)
    assert [int(a) for a in v] == [6457827717110365317, 3203168211198807973,
                                  9817491932198370423]


def test_lattice_start_geometry():
    s = synth.lattice_start(16, 0.70, 4, seed=3)
    L = s.box
    assert abs(16 * 16 * np.pi / (4 * L * L) - 0.70) < 1e-14
    assert np.all((s.x >= 0) & (s.x < L) & (s.y >= 0) & (s.y < L))
    sp = L / 16
    assert np.max(np.abs(s.x - (np.repeat(np.arange(16), 16) + 0.5) * sp)) <= 0.01 + 1e-15
    assert len(set(s.active.tolist())) == 4


@pytest.mark.parametrize("seed,row_shift,pair_shift", [(1, 0.05, 0.15), (5, 0.05, 0.15),
                                                        (8, 0.2, 0.0), (9, 0.2, 0.0)])
def test_staggered_start_geometry(seed, row_shift, pair_shift):
    """The staggered starts of the GPU tests are hard-disk configurations (every
    pair at least d apart, minimum image), with rows in close pairs (a gap
    below d in y) and pairs far apart (a gap above d) where pair_shift > 0."""
    s = synth.staggered_start(16, 0.5, 12, seed, row_shift=row_shift, pair_shift=pair_shift)
    L = s.box
    assert np.all((s.x >= 0) & (s.x < L) & (s.y >= 0) & (s.y < L))
    dx = np.abs(s.x[:, None] - s.x[None, :])
    dx = np.minimum(dx, L - dx)
    dy = np.abs(s.y[:, None] - s.y[None, :])
    dy = np.minimum(dy, L - dy)
    d2 = dx * dx + dy * dy
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 1.0
    assert len(set(s.active.tolist())) == 12
    if pair_shift > 0:
        rows = np.sort(s.y.reshape(16, 16)[0])  # column 0 (id = c m + r): one disk per row
        gaps = np.diff(np.concatenate([rows, rows[:1] + L]))
        assert (gaps < 1.0).any() and (gaps > 1.1).any()


# ------------------------------------------------------- closed forms


def _row_start(L, xs, yrow, d=1.0):
    """Disks along one row at height yrow, others absent."""
    x = np.array(xs, dtype=np.float64)
    y = np.full_like(x, yrow)
    return x, y


def test_single_row_closed_form():
    """Sec. 1, Eq. 1 on a 1D ring: each lift brings i to contact (dx = d) and
    the chain stalls when the remaining length is below the next gap.
    Positions are dyadic so the exact-rational walk is reproduced."""
    L, d, ell = 10.0, 1.0, 2.2
    xs = [0.5, 2.0, 3.25, 5.0, 6.5, 8.0]
    x, y = _row_start(L, xs, 5.0)
    r = O.run_leg(x, y, [0], L, ell, search=0)
    # exact walk
    pos = [Fraction(v) for v in xs]
    rem, m, t = Fraction(ell), 0, Fraction(0)
    lifts = []
    while True:
        nxt = (m + 1) % len(pos)
        gap = (pos[nxt] - pos[m]) % Fraction(L) - 1
        if gap < rem:
            pos[m] += gap
            t += gap
            rem -= gap
            lifts.append((m, nxt, t))
            m = nxt
        else:
            pos[m] += rem
            break
    assert r.active.tolist() == [m]
    assert [(e["i"], e["j"]) for e in r.log] == [(a, b) for a, b, _ in lifts]
    for e, (_, _, tt) in zip(r.log, lifts):
        assert abs(e["t"] - float(tt)) <= 4 * ulp(ell)
    for q in range(len(xs)):
        assert abs(r.x[q] - float(pos[q] % Fraction(L))) <= 4 * ulp(L)
    assert abs(r.t[m] - ell) <= 8 * ulp(ell)


def test_contact_distance_345():
    """Sec. 2.2 (time of flight as Alg. 5 computes it), Eq. 3: tau = dx - sqrt(d^2 - dy^2).
    dy = 0.6 gives b = 0.8 (a 3-4-5 triangle)."""
    L = 8.0
    x = np.array([1.0, 2.6, 6.0])
    y = np.array([4.0, 4.6, 1.0])
    lift, j, tau, _ = O.step(x, y, 0, 5.0, L, search=0)
    assert lift == 1 and j == 1
    assert abs(tau - 0.8) < 1e-15
    # after the lift the centres are at distance d
    r = O.run_leg(x, y, [0], L, 1.0, search=0)
    e = r.log[0]
    dx, dy = e["xj"] - e["xi"], 0.6
    assert abs(np.hypot(dx, dy) - 1.0) < 1e-14


def test_corridor_is_strict():
    """A disk at perpendicular distance exactly d is outside the corridor
    (Sec. 3.1: corridors of width 2 sigma, strict)."""
    L = 8.0
    x = np.array([1.0, 1.5, 6.0])
    y = np.array([4.0, 5.0, 1.0])
    lift, j, tau, _ = O.step(x, y, 0, 3.0, L, search=0)
    assert lift == 0 and tau == 3.0


def test_periodic_wrap_x_and_y():
    """Forward image in x, minimum image in y (the periodic reading)."""
    L = 9.0
    x = np.array([L - 0.3, 1.2, 4.0])
    y = np.array([0.3, L - 0.3, 4.0])
    lift, j, tau, _ = O.step(x, y, 0, 5.0, L, search=0)
    assert lift == 1 and j == 1
    assert abs(tau - (1.5 - 0.8)) < 1e-14
    r = O.run_leg(x, y, [0], L, 1.0, search=0)
    assert abs(r.log[0]["xi"] - 0.4) < 1e-14  # wrapped into [0, L)
    assert 0.0 <= r.x.min() and r.x.max() < L


def test_stall_without_candidates():
    """No candidate below D -> move by D and stall (Alg. 2 at the breakpoint)."""
    L = 9.0
    x = np.array([1.0, 4.0, 7.0])
    y = np.array([1.0, 4.0, 7.0])
    r = O.run_leg(x, y, [1], L, 0.75, search=0)
    assert r.lifts == 0
    assert r.x[1] == 4.75 and r.t[1] == 0.75 and r.active.tolist() == [1]


# ------------------------------------------------- cell scan == definition


@pytest.mark.parametrize("eta,seed", [(0.3, 1), (0.5, 2), (0.6, 3)])
def test_cell_scan_equals_all_pairs(eta, seed):
    """The cell scan with its stop rule returns the all-pairs argmin of Alg. 2."""
    if eta >= 0.55:
        s = synth.lattice_start(12, eta, 4, seed=seed)
    else:
        s = synth.rsa_start(120, eta, 4, seed=seed)
    rng = np.random.default_rng(seed)
    n = s.n
    for trial in range(300):
        i = int(rng.integers(n))
        D = float(rng.choice([0.05, 0.3, 1.0, 3.0, s.box / 2]))
        tag = (rng.random(n) < 0.1).astype(np.int8)
        tag[i] = 1
        a = O.step(s.x, s.y, i, D, s.box, search=0, tag=tag)
        for nc in {O.default_cells(s.box), 3, max(3, O.default_cells(s.box) // 2)}:
            b = O.step(s.x, s.y, i, D, s.box, search=1, nc=nc, tag=tag)
            assert a[:3] == b[:3], (trial, nc, a, b)


def test_cells_vs_all_pairs_full_legs():
    s = synth.rsa_start(150, 0.45, 6, seed=11)
    ra, _ = O.run_legs(s.x, s.y, s.active, s.box, 1.5, 4, search=0)
    rb, _ = O.run_legs(s.x, s.y, s.active, s.box, 1.5, 4, search=1)
    assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.t, rb.t)
    assert np.array_equal(ra.active, rb.active)


# ------------------------------------------------------------ invariants


def _min_pair_distance(x, y, L):
    dx = np.abs(x[:, None] - x[None, :])
    dx = np.minimum(dx, L - dx)
    dy = np.abs(y[:, None] - y[None, :])
    dy = np.minimum(dy, L - dy)
    r = np.hypot(dx, dy)
    np.fill_diagonal(r, np.inf)
    return r.min()


def _check_leg_invariants(x0, y, a0, r, L, ell, k):
    # no overlap (contact within rounding)
    assert _min_pair_distance(r.x, y, L) >= 1.0 - 1e-12
    # total displacement: every chain displaces its disks by ell in total
    disp = (r.x - x0) % L
    disp[disp > L / 2] -= L  # no disk moves backwards
    assert np.all(disp >= -1e-12)
    assert abs(disp.sum() - k * ell) <= 1e-12 * max(1.0, k * ell)
    # Remark 1: active (stalled) disks have t = ell, the others t < ell
    act = set(r.active.tolist())
    for c in range(k):
        assert abs(r.t[r.active[c]] - ell) <= (r.lifts_per_chain[c] + 2) * 2 * ulp(ell)
    others = np.array([q for q in range(len(x0)) if q not in act], dtype=int)
    assert np.all(r.t[others] < ell)
    # Remark 2 and Alg. 2: liftings in global-time order, positive t_j updates
    tprev = np.zeros(len(x0))
    last = -np.inf
    for e in r.log:
        assert e["t"] >= last
        last = e["t"]
        assert e["t"] >= tprev[e["j"]]
        assert e["t"] > tprev[e["j"]] or e["t"] == 0.0
        tprev[e["j"]] = e["t"]
        tprev[e["i"]] = e["t"]
        # contact at the lifting: |x' - x| = d (Eq. 1)
        dx = (e["xj"] - e["xi"]) % L
        dy = abs(y[e["j"]] - y[e["i"]])
        dy = min(dy, L - dy)
        assert abs(np.hypot(dx, dy) - 1.0) < 1e-12
    # per chain: the lift tau's plus the final stall move add up to ell
    for c in range(k):
        mine = [e for e in r.log if e["c"] == c]
        taus = [float(e["tau"]) for e in mine]
        i_end = int(r.active[c])
        x_act = float(mine[-1]["xj"]) if mine else float(x0[i_end])
        stall = (r.x[i_end] - x_act) % L
        assert abs(sum(taus) + stall - ell) <= 1e-12
        # lifting times are the running sums of the tau's
        run = 0.0
        for e in mine:
            run += float(e["tau"])
            assert abs(e["t"] - run) <= 1e-12


@pytest.mark.parametrize("seed", list(range(10)))
def test_invariants_lattice_config1(seed):
    """N=256 lattice at eta=0.70, 4 chains, ell=0.5, 8 legs."""
    s = synth.lattice_start(16, 0.70, 4, seed=seed)
    x, a = s.x.copy(), s.active.copy()
    for leg in range(8):
        r = O.run_leg(x, s.y, a, s.box, 0.5, leg=leg)
        _check_leg_invariants(x, s.y, a, r, s.box, 0.5, 4)
        x, a = r.x, r.active


@pytest.mark.parametrize("seed", [5, 6])
def test_invariants_random_2d(seed):
    """Non-lattice starts exercise the j+/j- corridors (cross-row lifts)."""
    s = synth.rsa_start(100, 0.5, 5, seed=seed)
    x, a = s.x.copy(), s.active.copy()
    cross = 0
    for leg in range(4):
        r = O.run_leg(x, s.y, a, s.box, 2.0, leg=leg)
        _check_leg_invariants(x, s.y, a, r, s.box, 2.0, 5)
        cross += int(np.sum(np.abs(s.y[r.log["j"]] - s.y[r.log["i"]]) > 0.5))
        x, a = r.x, r.active
    assert cross > 0


# -------------------------------------------------------- time reversal


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_time_reversal(seed):
    """Remark 3: running from the final lifted configuration with -v returns
    the initial configuration with the same liftings (reversed, at mirrored
    times). -v is realised by mirroring x -> L - x."""
    s = synth.rsa_start(80, 0.45, 3, seed=seed)
    L, ell = s.box, 1.3
    r = O.run_leg(s.x, s.y, s.active, L, ell, search=0)
    xm = (L - r.x) % L
    rr = O.run_leg(xm, s.y, r.active, L, ell, search=0)
    xback = (L - rr.x) % L
    d = np.abs(xback - s.x)
    d = np.minimum(d, L - d)
    assert d.max() < 1e-12
    assert rr.active.tolist() == s.active.tolist()
    fwd = sorted((int(e["i"]), int(e["j"]), float(e["t"])) for e in r.log)
    bwd = sorted((int(e["j"]), int(e["i"]), ell - float(e["t"])) for e in rr.log)
    assert [(a, b) for a, b, _ in fwd] == [(a, b) for a, b, _ in bwd]
    assert max(abs(a[2] - b[2]) for a, b in zip(fwd, bwd)) < 1e-12


# ------------------------------------------------------------- Lemma 2


def test_lemma2_alg4_equals_alg2():
    """Lemma 2: Alg. 4 (local times, chains one after another) that ends
    without a horizon violation gives the output of the global-time process."""
    ok = 0
    for seed in range(40):
        s = synth.rsa_start(60, 0.45, 3, seed=100 + seed)
        L, ell = s.box, 1.0
        g = O.run_leg(s.x, s.y, s.active, L, ell, search=0)
        rc, x4, t4, a4, log4 = O.run_alg4_leg(s.x, s.y, s.active, L, ell)
        if rc != 0:
            continue
        ok += 1
        dx = np.abs(x4 - g.x)
        dx = np.minimum(dx, L - dx)
        assert dx.max() < 1e-12
        assert np.max(np.abs(t4 - g.t)) < 1e-12
        assert a4.tolist() == g.active.tolist()
        assert sorted((e["c"], e["i"], e["j"]) for e in log4) == \
            sorted((e["c"], e["i"], e["j"]) for e in g.log)
    assert ok >= 10


def test_flag_zero_means_isolated_runs_compose():
    """When no two chains scan a common cell, running each chain alone (in
    chain order, on the shared state) is the global-time result (Lemma 2)."""
    seen = 0
    for seed in range(30):
        s = synth.lattice_start(24, 0.70, 3, seed=seed)
        L, ell = s.box, 0.5
        g = O.run_leg(s.x, s.y, s.active, L, ell)
        sets = [set(O.claim_set(s.x, s.y, int(a), L, ell).tolist()) for a in s.active]
        overlap = any(sets[p] & sets[q] for p in range(3) for q in range(p + 1, 3))
        assert g.flag == int(overlap)
        if g.flag == 0:
            seen += 1
            x, act = s.x.copy(), s.active.copy()
            for c in range(3):
                one = O.run_leg(x, s.y, act[c:c + 1], L, ell, search=0)
                x = one.x
            assert np.array_equal(x, g.x)
    assert seen >= 3


# ----------------------------------------------- literal Alg. 2 (global time)


def _tof(xi, yi, xj, yj, L, d=1.0):
    a = abs(yj - yi)
    a = min(a, L - a)
    if not a < d:
        return np.inf
    dx = (xj - xi) % L
    return max(0.0, dx - np.sqrt(d * d - a * a))


def literal_alg2(x, y, active, L, ell):
    """Alg. 2 as printed: at every event all active disks advance together to
    the event time. Independent of the oracle's lazy per-chain bookkeeping."""
    pos = np.array(x, dtype=float)
    act = [int(a) for a in active]
    now = 0.0
    lifts = []
    while True:
        best = (np.inf, None, None)
        aset = set(act)
        for c, i in enumerate(act):
            for j in range(len(pos)):
                if j in aset:
                    continue
                tau = _tof(pos[i], y[i], pos[j], y[j], L)
                if (tau, c, j) < (best[0], best[1] if best[1] is not None else 1 << 30,
                                  best[2] if best[2] is not None else 1 << 30):
                    best = (tau, c, j)
        dt = min(best[0], ell - now)
        for i in act:
            pos[i] = (pos[i] + dt) % L
        now += dt
        if best[0] < ell - (now - dt) and best[1] is not None and now < ell:
            c, j = best[1], best[2]
            lifts.append((c, act[c], j, now))
            act[c] = j
        else:
            break
    return pos, act, lifts


@pytest.mark.parametrize("seed", range(8))
def test_literal_global_time_algorithm(seed):
    """The oracle's global order with per-chain positions equals Alg. 2 read
    literally (within rounding): same liftings in the same order."""
    s = synth.rsa_start(40, 0.5, 4, seed=500 + seed)
    L, ell = s.box, 2.0
    g = O.run_leg(s.x, s.y, s.active, L, ell, search=0)
    pos, act, lifts = literal_alg2(s.x, s.y, s.active, L, ell)
    assert [(c, i, j) for c, i, j, _ in lifts] == \
        [(int(e["c"]), int(e["i"]), int(e["j"])) for e in g.log]
    assert max([abs(t - e["t"]) for (_, _, _, t), e in zip(lifts, g.log)] + [0]) < 1e-12
    dx = np.abs(pos - g.x)
    assert np.minimum(dx, L - dx).max() < 1e-12
    assert act == g.active.tolist()


@pytest.mark.parametrize("seed", [1, 2])
def test_claim_windows_only_change_the_flag(seed):
    """Cutting a leg into claim windows is scheduling only: the liftings,
    positions and local times of Alg. 2 are the same for every W."""
    s = synth.lattice_start(24, 0.70, 12, seed=seed)
    base = O.run_leg(s.x, s.y, s.active, s.box, 1.0, windows=1)
    for w in (2, 3, 8, 32):
        r = O.run_leg(s.x, s.y, s.active, s.box, 1.0, windows=w)
        assert np.array_equal(r.x, base.x) and np.array_equal(r.t, base.t)
        assert np.array_equal(r.active, base.active)
        assert np.array_equal(r.log, base.log)
    # chains far apart in time no longer meet once the leg is cut finely
    flags = [O.run_leg(s.x, s.y, s.active, s.box, 1.0, windows=w).flag for w in (1, 64)]
    assert flags[0] == 1
