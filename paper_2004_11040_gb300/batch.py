"""Batched replicas: many independent ECMC systems of uneven size in one
persistent launch, versus the same systems one at a time; and the autotuner
that picks the cell size and the legs per launch.

Replica recipe (the batched workload): N log-uniform in [1024, 65536] with
M = round(sqrt(N)), N := M^2; eta uniform in [0.60, 0.74]; k = M chains
(about sqrt(N)); ell = 1; seeded lattice starts.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import ecmc, synth


@dataclass
class Replica:
    start: synth.Start
    ell: float
    eta: float


def make_replicas(count: int, seed: int, n_range=(1024, 65536), eta_range=(0.60, 0.74),
                  ell: float = 1.0) -> list[Replica]:
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n_t = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        m = synth.lattice_m_for(int(n_t))
        eta = float(rng.uniform(*eta_range))
        out.append(Replica(synth.lattice_start(m, eta, m, seed=seed * 7919 + q), ell, eta))
    return out


def cells_for(start: synth.Start, factor: float) -> int:
    """Cells per side for a cell side of about factor * d (0 = default)."""
    if factor <= 1.0:
        return 0
    return max(3, int(start.box / (factor * start.d)))


def create(reps: list[Replica], cell_factor: float = 1.0, undo_cap: int = 256, stream=None):
    return [ecmc.System(r.start.x, r.start.y, r.start.active, r.start.box, r.ell,
                        cells_per_side=cells_for(r.start, cell_factor), undo_cap=undo_cap,
                        stream=stream) for r in reps]


def run_batched(systems, budget: int, legs_per_launch: int, stream=None):
    """All systems to `budget` liftings each; returns (liftings, device_ms, launches)."""
    batch = ecmc.ecmc_batch_create(stream)
    live = list(range(len(systems)))
    done = np.zeros(len(systems), dtype=np.int64)
    ms_total, launches = 0.0, 0
    try:
        while live:
            lifts, legs, ms = ecmc.ecmc_batch_run(batch, [systems[q].ctx for q in live],
                                                  legs_per_launch, [budget - done[q] for q in live])
            ms_total += ms
            launches += 1
            for q, nl in zip(live, lifts):
                done[q] += int(nl)
            live = [q for q in live if done[q] < budget]
    finally:
        ecmc.ecmc_batch_destroy(batch)
    return int(done.sum()), ms_total, launches


def run_plain(systems, budget: int, legs_per_launch: int):
    """One system at a time through ecmc_run_to_breakpoint."""
    total, ms_total, launches = 0, 0.0, 0
    for sysm in systems:
        got = 0
        while got < budget:
            b = sysm.stats()
            sysm.run(legs_per_launch, event_budget=budget - got)
            e = sysm.stats()
            got += e["liftings"] - b["liftings"]
            ms_total += e["device_ms"] - b["device_ms"]
            launches += 1
        total += got
    return total, ms_total, launches


# ----------------------------------------------------------------- autotuner

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ecmc_gb300_autotune.json")


def _key(reps: list[Replica]) -> str:
    ns = sorted(r.start.n for r in reps)
    return f"n{ns[0]}-{ns[-1]}_r{len(reps)}"


def autotune(reps: list[Replica], trial_budget: int = 20_000,
             cell_factors=(1.0, 1.5), legs_options=(4, 16, 64), cache: str | None = CACHE,
             stream=None) -> dict:
    """Tries every (cell size, legs per launch) on a sample of the replicas and
    keeps the fastest by liftings per device second; the choice is cached per
    workload key. Warps per chain is 1: an FP64 warp instruction costs the same
    whatever the number of active lanes on this GPU, so more warps per chain
    buy no throughput."""
    key = _key(reps)
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                got = json.load(f).get(key)
            if got:
                return got
        except Exception:
            pass
    sample = reps[: min(len(reps), 64)]
    best = None
    trials = []
    for cf in cell_factors:
        systems = create(sample, cf, stream=stream)
        try:
            for legs in legs_options:
                lifts, ms, _ = run_batched(systems, trial_budget, legs, stream=stream)
                rate = lifts / (ms / 1e3) if ms > 0 else 0.0
                trials.append({"cell_factor": cf, "legs_per_launch": legs, "liftings_per_s": rate})
                if best is None or rate > best["liftings_per_s"]:
                    best = dict(trials[-1])
        finally:
            for s in systems:
                s.close()
    best["trials"] = trials
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    data = json.load(f)
            data[key] = best
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
        except Exception:
            pass
    return best


def bench_batched(count: int = 512, budget: int = 1_000_000, plain_sample: int = 16,
                  seed: int = 0, tune: bool = True, stream=None) -> dict:
    """Batched throughput of `count` replicas to `budget` liftings each, and the
    one-at-a-time throughput on the first `plain_sample` of them."""
    reps = make_replicas(count, seed)
    choice = autotune(reps, stream=stream) if tune else {"cell_factor": 1.0,
                                                          "legs_per_launch": 16}
    t0 = time.perf_counter()
    systems = create(reps, choice["cell_factor"], stream=stream)
    t_create = time.perf_counter() - t0
    try:
        lifts, ms, launches = run_batched(systems, budget, choice["legs_per_launch"], stream)
    finally:
        for s in systems:
            s.close()
    plain_sys = create(reps[:plain_sample], choice["cell_factor"], stream=stream)
    try:
        p_lifts, p_ms, p_launches = run_plain(plain_sys, budget, choice["legs_per_launch"])
    finally:
        for s in plain_sys:
            s.close()
    batched = lifts / (ms / 1e3)
    plain = p_lifts / (p_ms / 1e3)
    return {"replicas": count, "budget_per_replica": budget, "liftings": lifts,
            "device_ms": ms, "launches": launches, "liftings_per_s": batched,
            "plain_sample": plain_sample, "plain_liftings_per_s": plain,
            "batched_over_plain": batched / plain if plain else None,
            "create_s": t_create, "autotune": {k: v for k, v in choice.items() if k != "trials"}}
