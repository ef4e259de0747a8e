"""The oracle's per-window conflict flags (W > 1 claim windows per leg),
pinned against an independent helper (tests/window_claims.py) and against
Lemma 2 window by window: where a window's flag is 0, the chains run alone
through it one after another, from the window-start state, give the global
state at the window's end bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import synth

import window_claims as WC

STARTS = {
    "lattice": lambda seed: synth.lattice_start(32, 0.70, 5, seed=seed),
    "rsa": lambda seed: synth.rsa_start(300, 0.45, 5, seed=seed),
    "staggered": lambda seed: synth.staggered_start(20, 0.55, 5, seed=seed, row_shift=0.05,
                                                    pair_shift=0.15),
}


def leg(s, W, ell=1.0):
    nc = O.default_cells(s.box, s.d)
    r = O.run_leg(s.x, s.y, s.active, s.box, ell, d=s.d, nc=nc, windows=W)
    return r, WC.Geometry(s.box, s.d, nc)


@pytest.mark.parametrize("kind", sorted(STARTS))
@pytest.mark.parametrize("W", [2, 5, 16])
def test_window_flags_equal_claim_set_overlap(kind, W):
    zeros = ones = 0
    for seed in range(4):
        s = STARTS[kind](seed)
        r, g = leg(s, W)
        want = WC.window_flags(g, s.x, s.y, s.active, 1.0, W, r.log)
        assert r.wflags.tolist() == want, (seed, r.wflags.tolist(), want)
        assert r.flag == int(any(want))
        zeros += want.count(0)
        ones += want.count(1)
    # both outcomes occur, so neither side can pass by answering one of them
    assert zeros > 0 and ones > 0, (zeros, ones)


@pytest.mark.parametrize("kind", sorted(STARTS))
@pytest.mark.parametrize("W", [2, 5, 16])
def test_flag_zero_windows_compose(kind, W):
    """Lemma 2 window by window."""
    checked = 0
    for seed in range(4):
        s = STARTS[kind](seed)
        r, g = leg(s, W)
        for w in range(W):
            if r.wflags[w]:
                continue
            x, t, act = WC.compose_window(g, s.x, s.y, s.active, 1.0, W, r.log, w)
            if w + 1 < W:
                ex, et, ea, _ = WC.replay(s.x, s.active, 1.0, r.log, WC.window_end(1.0, W, w))
            else:
                ex, et, ea = r.x, r.t, r.active
            assert np.array_equal(x, ex), (seed, w)
            assert np.array_equal(t, et), (seed, w)
            assert act.tolist() == ea.tolist(), (seed, w)
            checked += 1
    assert checked > 0


def test_a_planted_mistake_is_caught():
    """The helper notices a flag computed from the leg's start state instead
    of the window's (a plausible slip): on this leg the two disagree."""
    s = STARTS["lattice"](0)
    W = 5
    r, g = leg(s, W)
    from_start = []
    for w in range(W):
        # every window's isolated runs from the leg's start state
        owner, hit = {}, 0
        for c, a in enumerate(s.active):
            xs, ts = s.x.copy(), np.zeros_like(s.x)
            claims, _, _ = WC.run_alone(g, xs, s.y, ts, int(a), 1.0, WC.window_end(1.0, W, w))
            for q in claims:
                if owner.setdefault(q, c) != c:
                    hit = 1
        from_start.append(hit)
    assert from_start != r.wflags.tolist()
