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


# ---- constraint-graph contexts in batches (their own persistent kernel)

def test_graph_batch_replicas_equal_oracle_and_alone():
    """Graph-mode systems of uneven size in one batch launch: each equals the
    oracle's graph-mode legs (search = 2: positions, local times, liftings
    and flags) and the same system run alone."""
    starts = _mixed_starts()
    legs = 4
    systems = [ecmc.System(s.x, s.y, s.active, s.box, ell, log=True, graph=True)
               for s, ell in starts]
    batch = ecmc.ecmc_batch_create()
    lifts, done, ms = ecmc.ecmc_batch_run(batch, [sy.ctx for sy in systems], legs)
    ecmc.ecmc_batch_destroy(batch)
    assert (done == legs).all() and ms > 0
    for (s, ell), sy, nl in zip(starts, systems, lifts):
        x, y, t, a = sy.positions()
        last, per_leg = O.run_legs(s.x, s.y, s.active, s.box, ell, legs, search=2)
        assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
        assert np.array_equal(a, last.active)
        assert nl == sum(r.lifts for r in per_leg)
        st = sy.stats()
        assert st["conflict_legs"] == sum(r.flag for r in per_leg)
        assert st["conflict_windows"] == sum(int(r.wflags.sum()) for r in per_leg)
        assert st["horizon_asserts"] == 0 and st["order_errors"] == 0
        log = sy.liftings()
        olog = np.concatenate([r.log for r in per_leg])
        key = lambda L: L[np.lexsort((np.arange(len(L)), L["c"], L["leg"]))]
        a_, b_ = key(olog), key(log)
        for f in ("leg", "c", "i", "j", "t", "tau", "xi", "xj"):
            assert np.array_equal(a_[f], b_[f]), f
        alone = ecmc.System(s.x, s.y, s.active, s.box, ell, graph=True)
        alone.run(legs)
        ax, _, at, aa = alone.positions()
        alone.close()
        assert np.array_equal(ax, x) and np.array_equal(at, t) and np.array_equal(aa, a)
        sy.close()


def test_graph_batch_budgets_and_windows():
    """Budgets stop each graph replica at a breakpoint, with claim windows
    (W = 3, the same for all); consecutive batch launches continue where the
    last one stopped."""
    starts = _mixed_starts()[:4]
    systems = [ecmc.System(s.x, s.y, s.active, s.box, ell, graph=True, windows=3)
               for s, ell in starts]
    budgets = [50, 1, 400, 10_000_000]
    batch = ecmc.ecmc_batch_create()
    lifts, legs, _ = ecmc.ecmc_batch_run(batch, [sy.ctx for sy in systems], 12, budgets)
    for (s, ell), sy, b, nl, ng in zip(starts, systems, budgets, lifts, legs):
        _, per_leg = O.run_legs(s.x, s.y, s.active, s.box, ell, 12, search=2, windows=3)
        cum = np.cumsum([r.lifts for r in per_leg])
        stop = int(np.searchsorted(cum, b) + 1) if cum[-1] >= b else 12
        assert ng == stop and nl == cum[stop - 1]
    # a second launch: 2 more legs each
    ecmc.ecmc_batch_run(batch, [sy.ctx for sy in systems], 2)
    ecmc.ecmc_batch_destroy(batch)
    for (s, ell), sy in zip(starts, systems):
        n = sy.stats()["legs"]
        last, _ = O.run_legs(s.x, s.y, s.active, s.box, ell, n, search=2, windows=3)
        x, _, t, a = sy.positions()
        assert np.array_equal(x, last.x) and np.array_equal(t, last.t)
        assert np.array_equal(a, last.active)
        sy.close()


def test_batch_rejects_mixed_searches():
    s = synth.lattice_start(16, 0.7, 4, seed=1)
    a = ecmc.System(s.x, s.y, s.active, s.box, 0.5)
    g = ecmc.System(s.x, s.y, s.active, s.box, 0.5, graph=True)
    batch = ecmc.ecmc_batch_create()
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.ecmc_batch_run(batch, [a.ctx, g.ctx], 1)
    assert e.value.code == ecmc.ECMC_EINVAL
    ecmc.ecmc_batch_destroy(batch)
    a.close()
    g.close()
