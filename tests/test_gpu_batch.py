"""Batches: independent systems of uneven size advanced by one persistent
launch. Each replica must be, bit for bit, what the oracle gives for it
alone, and what the same system gives when run alone on the GPU."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import ecmc, synth

pytestmark = pytest.mark.gpu


def _mixed_starts():
    rng = np.random.default_rng(2024)
    out = []
    for q in range(6):
        m = int(rng.integers(8, 40))
        eta = float(rng.uniform(0.60, 0.74))
        k = max(1, int(round(m * float(rng.uniform(0.3, 1.5)))))
        out.append((synth.lattice_start(m, eta, k, seed=100 + q), float(rng.uniform(0.4, 1.5))))
    out.append((synth.rsa_start(200, 0.45, 5, seed=7), 1.2))
    return out


def test_batch_replicas_equal_oracle_and_alone():
    starts = _mixed_starts()
    legs = 4
    systems = [ecmc.System(s.x, s.y, s.active, s.box, ell, log=True) for s, ell in starts]
    batch = ecmc.ecmc_batch_create()
    lifts, done, ms = ecmc.ecmc_batch_run(batch, [sy.ctx for sy in systems], legs)
    ecmc.ecmc_batch_destroy(batch)
    assert (done == legs).all() and ms > 0
    for (s, ell), sy, nl in zip(starts, systems, lifts):
        x, y, t, a = sy.positions()
        last, per_leg = O.run_legs(s.x, s.y, s.active, s.box, ell, legs)
        assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
        assert np.array_equal(a, last.active)
        assert nl == sum(r.lifts for r in per_leg)
        st = sy.stats()
        assert st["conflict_legs"] == sum(r.flag for r in per_leg)
        assert st["horizon_asserts"] == 0 and st["order_errors"] == 0
        alone = ecmc.System(s.x, s.y, s.active, s.box, ell)
        alone.run(legs)
        ax, _, at, aa = alone.positions()
        alone.close()
        assert np.array_equal(ax, x) and np.array_equal(at, t) and np.array_equal(aa, a)
        sy.close()


def test_batch_budgets_stop_each_replica_at_a_breakpoint():
    starts = _mixed_starts()[:4]
    systems = [ecmc.System(s.x, s.y, s.active, s.box, ell) for s, ell in starts]
    budgets = [50, 1, 400, 10_000_000]
    batch = ecmc.ecmc_batch_create()
    lifts, legs, _ = ecmc.ecmc_batch_run(batch, [sy.ctx for sy in systems], 12, budgets)
    ecmc.ecmc_batch_destroy(batch)
    for (s, ell), sy, b, nl, ng in zip(starts, systems, budgets, lifts, legs):
        # the oracle's cumulative liftings decide the stopping leg
        _, per_leg = O.run_legs(s.x, s.y, s.active, s.box, ell, 12)
        cum = np.cumsum([r.lifts for r in per_leg])
        stop = int(np.searchsorted(cum, b) + 1) if cum[-1] >= b else 12
        assert ng == stop and nl == cum[stop - 1]
        sy.close()


def test_single_context_leg_flags_through_persistent_kernel():
    s = synth.lattice_start(24, 0.7, 6, seed=3)
    sy = ecmc.System(s.x, s.y, s.active, s.box, 0.6)
    flags, done = sy.run(5)
    _, per_leg = O.run_legs(s.x, s.y, s.active, s.box, 0.6, 5)
    assert flags.tolist() == [r.flag for r in per_leg]
    sy.close()
