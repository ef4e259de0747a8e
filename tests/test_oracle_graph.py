"""Pins for the oracle's constraint graph G(3) (Sec. 3.1) and its graph-mode
leg, against facts the paper and the geometry fix.

- The lattice starts have a closed-form graph: the centre arrow of every disk
  is the next disk of its row, and the side corridors are empty (adjacent rows
  are more than d apart in y).
- An arrow is the nearest disk ahead, by forward distance in x, in its
  corridor (Sec. 3.1 says the lifting partners are the closest disks of the
  three corridors); the oracle defines it by least time of flight.
- Arrows do not change between breakpoints (Sec. 3.1: disks closer than d in y
  cannot hop over one another).
- Every lifting of the all-pairs Alg. 2 runs along an arrow (the validation of
  Sec. 4: the liftings of cell ECMC are all accounted for in the graph).
- A graph-mode leg equals the all-pairs leg, and its flag is the overlap of
  the disks that isolated chains read, built here from single-chain all-pairs
  runs and the graph.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import synth


def _corridor(yi, yj, L, d=1.0):
    dy = yj - yi
    dy = dy - L * np.round(dy / L)  # minimum image in [-L/2, L/2]
    a = abs(dy)
    if not a < d:
        return -1
    if a < 0.5 * d:
        return 0
    return 1 if dy > 0 else 2


@pytest.mark.parametrize("m,eta,seed", [(16, 0.70, 0), (24, 0.72, 3), (12, 0.74, 5)])
def test_lattice_graph_is_the_row_ring(m, eta, seed):
    """Lattice start (site (c, r) = disk c*m + r): the centre arrow of a disk
    is the disk of the next column in its row, the side corridors are empty."""
    s = synth.lattice_start(m, eta, 4, seed=seed)
    g = O.graph3(s.x, s.y, s.box, search=0)
    ids = np.arange(m * m)
    col, row = ids // m, ids % m
    nxt = ((col + 1) % m) * m + row
    assert np.array_equal(g[:, 0], nxt)
    assert np.all(g[:, 1] == -1) and np.all(g[:, 2] == -1)


@pytest.mark.parametrize("n,eta,seed", [(150, 0.3, 1), (300, 0.5, 2), (400, 0.45, 4)])
def test_cell_scan_builds_the_same_graph(n, eta, seed):
    s = synth.rsa_start(n, eta, 2, seed=seed)
    ref = O.graph3(s.x, s.y, s.box, search=0)
    nc0 = O.default_cells(s.box)
    for nc in {nc0, 3, max(3, nc0 // 2)}:
        assert np.array_equal(O.graph3(s.x, s.y, s.box, nc=nc, search=1), ref), nc
    ids = np.array([0, n - 1, n // 2, 7], dtype=np.int32)
    assert np.array_equal(O.graph3(s.x, s.y, s.box, search=1, ids=ids), ref[ids])


def test_outdegree_three_except_small_systems():
    """Sec. 3.1: G(3) has outdegree three for all disks except in small
    systems, where corridors may be empty."""
    s = synth.rsa_start(400, 0.5, 2, seed=9)
    g = O.graph3(s.x, s.y, s.box)
    assert np.all(g >= 0)
    # a 3 x 3 lattice in a box of side ~3.2: only the own row is within d
    t = synth.lattice_start(3, 0.70, 1, seed=1)
    gt = O.graph3(t.x, t.y, t.box)
    assert np.all(gt[:, 0] >= 0) and np.all(gt[:, 1:] == -1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_arrow_is_nearest_ahead_in_its_corridor(seed):
    """Independent characterisation: the arrow is the disk of least forward
    distance in x among those of its corridor, and it lies in that corridor."""
    s = synth.rsa_start(250, 0.5, 2, seed=40 + seed)
    L = s.box
    g = O.graph3(s.x, s.y, L)
    for i in range(s.n):
        best = [None, None, None]
        for j in range(s.n):
            if j == i:
                continue
            kc = _corridor(s.y[i], s.y[j], L)
            if kc < 0:
                continue
            dx = (s.x[j] - s.x[i]) % L
            if best[kc] is None or dx < best[kc][0]:
                best[kc] = (dx, j)
        for kc in range(3):
            want = -1 if best[kc] is None else best[kc][1]
            assert g[i, kc] == want, (i, kc)


@pytest.mark.parametrize("seed", [5, 6])
def test_arrows_unchanged_between_breakpoints(seed):
    """Sec. 3.1: after any number of legs along +x the graph rebuilt from the
    new configuration is the graph of the old one."""
    s = synth.rsa_start(200, 0.5, 6, seed=seed)
    g0 = O.graph3(s.x, s.y, s.box)
    r, _ = O.run_legs(s.x, s.y, s.active, s.box, 3.0, 5, search=0)
    assert not np.array_equal(r.x, s.x)
    assert np.array_equal(O.graph3(r.x, s.y, s.box), g0)


@pytest.mark.parametrize("seed", [7, 8])
def test_every_lifting_runs_along_an_arrow(seed):
    """Sec. 4 validation: every lifting i -> j of (all-pairs) Alg. 2 is an
    arrow of the graph of the starting configuration."""
    s = synth.rsa_start(300, 0.5, 8, seed=seed)
    g = O.graph3(s.x, s.y, s.box)
    _, legs = O.run_legs(s.x, s.y, s.active, s.box, 2.0, 4, search=0)
    n = 0
    for lg in legs:
        for e in lg.log:
            assert int(e["j"]) in g[int(e["i"])].tolist()
            n += 1
    assert n > 100


@pytest.mark.parametrize("kind,seed", [("rsa", 11), ("rsa", 12), ("lattice", 13)])
def test_graph_leg_equals_all_pairs_leg(kind, seed):
    if kind == "rsa":
        s = synth.rsa_start(220, 0.5, 10, seed=seed)
        ell, legs = 1.5, 4
    else:
        s = synth.lattice_start(16, 0.70, 12, seed=seed)
        ell, legs = 1.0, 4
    ra, la = O.run_legs(s.x, s.y, s.active, s.box, ell, legs, search=0)
    for w in (1, 3):
        rb, lb = O.run_legs(s.x, s.y, s.active, s.box, ell, legs, search=2, windows=w)
        assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.t, rb.t)
        assert np.array_equal(ra.active, rb.active)
        for a, b in zip(la, lb):
            assert np.array_equal(a.log, b.log)


def _vertex_claims(x, y, a0, L, ell, graph):
    """Disks an isolated chain reads: its active disks (start and every lift
    target) and their arrows, from a single-chain all-pairs run."""
    one = O.run_leg(x, y, [a0], L, ell, search=0)
    visited = [a0] + [int(e["j"]) for e in one.log]
    out = set(visited)
    for v in visited:
        out.update(int(j) for j in graph[v] if j >= 0)
    return out


def test_graph_flag_is_overlap_of_read_disks():
    flags = []
    for seed in range(16):
        if seed % 2:
            s = synth.rsa_start(160, 0.5, 3, seed=100 + seed)
        else:
            s = synth.lattice_start(12, 0.70, 4, seed=100 + seed)
        L, ell = s.box, 0.8
        g = O.graph3(s.x, s.y, L)
        r = O.run_leg(s.x, s.y, s.active, L, ell, search=2)
        sets = [_vertex_claims(s.x, s.y, int(a), L, ell, g) for a in s.active]
        k = len(sets)
        overlap = any(sets[p] & sets[q] for p in range(k) for q in range(p + 1, k))
        assert r.flag == int(overlap), seed
        flags.append(r.flag)
        if r.flag == 0:
            # Lemma 2: the chains run one after another give the same result
            x, act = s.x.copy(), s.active.copy()
            for c in range(k):
                x = O.run_leg(x, s.y, act[c:c + 1], L, ell, search=0).x
            assert np.array_equal(x, r.x)
    assert 0 < sum(flags) < len(flags)
