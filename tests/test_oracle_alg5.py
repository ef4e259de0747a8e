"""Exhaustive interleavings of Alg. 5 (sequential-consistency model) pin the oracle.

Lemma 3's method: every state reachable by any interleaving of two threads'
shared-memory accesses is enumerated; every "terminate" state must equal the global-time
result (Alg. 2, the oracle). The paper's own test suites (SequentialC4/C5)
are not available, so seeded random 4- and 5-disk configurations in a box of
side 4 stand in for them. The mutation test writes a lifted disk's position
before its local time (the order Remark 11 warns against) and must produce a
terminate state that the correct program never reaches.
"""
import numpy as np
import pytest

from oracle import oracle as O

from alg5_model import explore

L_BOX = 4.0


def tiny(seed, n=4, L=L_BOX):
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    while len(xs) < n:
        cx, cy = rng.random() * L, rng.random() * L * 0.5 + L * 0.25
        ok = True
        for px, py in zip(xs, ys):
            dx = abs(px - cx)
            dx = min(dx, L - dx)
            dy = abs(py - cy)
            dy = min(dy, L - dy)
            if dx * dx + dy * dy < 1:
                ok = False
        if ok:
            xs.append(cx)
            ys.append(cy)
    act = rng.choice(n, 2, replace=False)
    ell = float(rng.uniform(0.5, 2.5))
    return np.array(xs), np.array(ys), act.astype(np.int32), ell


def _matches(state, g):
    return np.array_equal(np.array(state[0]), g.x) and np.array_equal(np.array(state[1]), g.t)


@pytest.mark.parametrize("n,seeds", [(4, range(0, 40)), (5, range(100, 112))])
def test_every_terminate_state_equals_global_time(n, seeds):
    n_term = 0
    for seed in seeds:
        x, y, a, ell = tiny(seed, n=n)
        g = O.run_leg(x, y, a, L_BOX, ell, search=0)
        terms, n_states, aborted, _ = explore(x, y, a, L_BOX, ell)
        assert n_states > 50  # a non-trivial enumeration
        for s in terms:
            assert _matches(s, g), seed
            # final active disks: thread c holds chain c's stalled disk
            assert [t[1] for t in s[3]] == g.active.tolist()
        n_term += len(terms) > 0
    assert n_term >= len(list(seeds)) // 3


def test_absorbing_when_no_necklace():
    """Lemma 3: from every reachable state an absorbing state (terminate or
    abort) can be reached, for configurations without necklaces."""
    good = 0
    for seed in range(0, 16):
        x, y, a, ell = tiny(seed)
        _, _, _, absorbing = explore(x, y, a, L_BOX, ell)
        good += absorbing
    assert good >= 14


def test_position_before_local_time_creates_spurious_state():
    """Remark 11: with t_i and x_i updated in the other order a thread can read
    the moved position with the old local time; some interleaving then ends in
    a terminate state that the correct program never reaches."""
    x, y, a, ell = tiny(11)
    g = O.run_leg(x, y, a, L_BOX, ell, search=0)
    terms, _, _, _ = explore(x, y, a, L_BOX, ell)
    mterms, _, _, _ = explore(x, y, a, L_BOX, ell, late_time=True)
    assert all(_matches(s, g) for s in terms)
    assert any(not _matches(s, g) for s in mterms)
