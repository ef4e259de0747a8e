"""The multicore CPU baseline (Alg. 5 on host threads). It is not an oracle,
but its single-thread runs are pinned: one chain equals the oracle over several
legs, and sequential chains without a horizon violation equal Alg. 2 (Lemma 2)."""
import numpy as np

from oracle import alg5
from oracle import oracle as O
from paper_2004_11040_gb300 import synth


def test_one_chain_one_thread_equals_oracle():
    s = synth.lattice_start(16, 0.70, 1, seed=4)
    got = alg5.run(s.x, s.y, s.active, s.box, 0.5, 6, threads=1)
    last, legs = O.run_legs(s.x, s.y, s.active, s.box, 0.5, 6)
    assert got.violations == 0
    assert got.lifts == sum(r.lifts for r in legs)
    assert np.array_equal(got.x, last.x)
    assert np.array_equal(got.active, last.active)


def test_one_chain_2d_random_start_equals_oracle():
    s = synth.rsa_start(300, 0.45, 1, seed=8)
    got = alg5.run(s.x, s.y, s.active, s.box, 1.5, 4, threads=1)
    last, legs = O.run_legs(s.x, s.y, s.active, s.box, 1.5, 4)
    assert got.lifts == sum(r.lifts for r in legs)
    assert np.array_equal(got.x, last.x)


def test_sequential_chains_without_violation_equal_alg2():
    matched = 0
    for seed in range(8):
        s = synth.lattice_start(16, 0.70, 4, seed=seed)
        got = alg5.run(s.x, s.y, s.active, s.box, 0.5, 1, threads=1)
        if got.violations:
            continue
        r = O.run_leg(s.x, s.y, s.active, s.box, 0.5, log=False)
        assert got.lifts == r.lifts
        assert np.array_equal(got.x, r.x)
        assert np.array_equal(got.active, r.active)
        matched += 1
    assert matched >= 2


def test_threads_run_and_keep_disks_in_box():
    s = synth.lattice_start(64, 0.72, 64, seed=1)
    got = alg5.run(s.x, s.y, s.active, s.box, 1.0, 3, threads=4)
    assert got.lifts > 0 and got.seconds > 0
    assert np.all((got.x >= 0) & (got.x < s.box))
    assert len(set(got.active.tolist())) == 64
