"""The batched runner's and the autotuner's host logic on the CPU
(paper_2004_11040_gb300/batch.py), with the library replaced by a fake: the
launch loop runs every system to its budget, the tuner tries every (cells,
search, legs) combination once (graph mode with one cell size), keeps the
fastest, records every trial and caches the choice per GPU, library build and
workload. The device side is tests/test_gpu_batch.py and test_gpu_serving.py."""
import numpy as np
import pytest

from paper_2004_11040_gb300 import batch

PER_LEG = 5  # liftings per chain and leg in the fake


class FakeSystem:
    def __init__(self, k, rate):
        self.ctx = id(self)
        self.k = k
        self.rate = rate  # liftings per device ms
        self.lifts = 0
        self.closed = False

    def stats(self):
        return {"liftings": self.lifts, "device_ms": self.lifts / self.rate, "row_windows": 0}

    def close(self):
        self.closed = True


class FakeBatchLib:
    def __init__(self):
        self.by_ctx = {}
        self.launches = []

    def create(self):
        return "b"

    def destroy(self, b):
        pass

    def run(self, b, ctxs, max_legs, budgets=None):
        lifts = np.zeros(len(ctxs), dtype=np.int64)
        legs = np.zeros(len(ctxs), dtype=np.int32)
        ms = 0.0
        for q, c in enumerate(ctxs):
            s = self.by_ctx[c]
            for _ in range(max_legs):
                lifts[q] += PER_LEG * s.k
                legs[q] += 1
                if budgets is not None and lifts[q] >= budgets[q]:
                    break
            s.lifts += int(lifts[q])
            ms = max(ms, lifts[q] / s.rate)
        self.launches.append((len(ctxs), max_legs))
        return lifts, legs, ms


# liftings per device ms of each trial setting in the fake: one clear winner
RATE = {("lattice", "row"): 100.0, ("default", "row"): 60.0, ("lattice", "general"): 40.0,
        ("default", "general"): 30.0, ("lattice", "graph"): 150.0}
LEG_BONUS = {4: 1.0, 16: 1.2, 64: 0.9}


@pytest.fixture
def fake(monkeypatch):
    lib = FakeBatchLib()
    made = []

    def create(sample, cells, stream=None, rowpass=True, graph=False):
        search = "graph" if graph else ("row" if rowpass else "general")
        out = []
        for r in sample:
            s = FakeSystem(r.start.k, RATE[(cells, search)])
            s.setting = (cells, search)
            lib.by_ctx[s.ctx] = s
            out.append(s)
        made.append((cells, search, out))
        return out

    real_run_batched = batch.run_batched

    def run_batched(systems, budget, legs, stream=None):
        lifts, ms, launches = real_run_batched(systems, budget, legs, stream=stream)
        return lifts, ms / LEG_BONUS[legs], launches

    monkeypatch.setattr(batch, "create", create)
    monkeypatch.setattr(batch.ecmc, "ecmc_batch_create", lambda stream=None: lib.create())
    monkeypatch.setattr(batch.ecmc, "ecmc_batch_destroy", lib.destroy)
    monkeypatch.setattr(batch.ecmc, "ecmc_batch_run", lib.run)
    monkeypatch.setattr(batch, "_hardware_key", lambda: "GPU_lib1")
    return lib, made, run_batched


def test_run_batched_takes_every_system_to_its_budget(fake):
    lib, made, _ = fake
    systems = [FakeSystem(k, 10.0) for k in (3, 8, 20, 50)]
    for s in systems:
        lib.by_ctx[s.ctx] = s
    total, ms, launches = batch.run_batched(systems, budget=1000, legs_per_launch=4)
    for s in systems:
        # stops at the first leg end at or past the budget
        assert 1000 <= s.lifts < 1000 + PER_LEG * s.k
    assert total == sum(s.lifts for s in systems)
    assert launches == len(lib.launches) and launches >= 2
    # systems that are done leave the launches
    assert [n for n, _ in lib.launches] == sorted([n for n, _ in lib.launches], reverse=True)


def test_autotune_keeps_the_fastest_and_records_every_trial(fake, tmp_path, monkeypatch):
    lib, made, run_batched = fake
    monkeypatch.setattr(batch, "run_batched", run_batched)
    reps = batch.make_replicas(12, seed=1, n_range=(1024, 4096))
    cache = str(tmp_path / "tune.json")
    got = batch.autotune(reps, trial_budget=500, cache=cache)
    # every combination once; graph mode with the first cell size only
    settings = [(t["cells"], t["search"], t["legs_per_launch"]) for t in got["trials"]]
    want = [(c, s, l) for s in ("row", "general", "graph") for c in ("lattice", "default")
            if s != "graph" or c == "lattice" for l in (4, 16, 64)]
    assert sorted(settings) == sorted(want) and len(settings) == len(set(settings))
    # the chains a warp advances: one in the cell scans, one per thread in graph mode
    assert {(t["search"], t["chains_per_warp"]) for t in got["trials"]} == \
           {("row", 1), ("general", 1), ("graph", 32)}
    best = max(got["trials"], key=lambda t: t["liftings_per_s"])
    assert (got["cells"], got["search"], got["legs_per_launch"]) == \
           (best["cells"], best["search"], best["legs_per_launch"]) == ("lattice", "graph", 16)
    assert all(s.closed for _, _, out in made for s in out)  # trial systems freed
    assert got["key"].startswith("GPU_lib1_n")


def test_autotune_cache_is_keyed_by_gpu_build_and_workload(fake, tmp_path, monkeypatch):
    lib, made, run_batched = fake
    monkeypatch.setattr(batch, "run_batched", run_batched)
    reps = batch.make_replicas(12, seed=1, n_range=(1024, 4096))
    cache = str(tmp_path / "tune.json")
    first = batch.autotune(reps, trial_budget=500, cache=cache)
    n_made = len(made)
    again = batch.autotune(reps, trial_budget=500, cache=cache)
    assert again == first and len(made) == n_made  # served from the cache: no trials
    # another library build: tried again
    monkeypatch.setattr(batch, "_hardware_key", lambda: "GPU_lib2")
    other = batch.autotune(reps, trial_budget=500, cache=cache)
    assert len(made) > n_made and other["key"] != first["key"]
    # another workload: tried again
    n_made = len(made)
    batch.autotune(reps[:6], trial_budget=500, cache=cache)
    assert len(made) > n_made
