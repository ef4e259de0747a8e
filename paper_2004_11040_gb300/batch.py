"""Batched replicas: many independent ECMC systems of uneven size in one
persistent launch, versus the same systems one at a time; and the autotuner
that picks the cell size, the parallel pass and the legs per launch.

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


def cells_for(start: synth.Start, cells) -> int:
    """Cells per side: "lattice" -- one cell per lattice site (cells aligned
    with the start lattice, so that every row of disks lies inside one cell
    row), "default" -- the library's choice (the smallest cells of side >= d),
    or a number f > 1 for cells of side about f * d."""
    if cells == "lattice":
        return int(start.m) if start.m > 0 else 0
    if cells == "default" or float(cells) <= 1.0:
        return 0
    return max(3, int(start.box / (float(cells) * start.d)))


def create(reps: list[Replica], cells="lattice", undo_cap: int = 256, stream=None,
           rowpass: bool = True, graph: bool = False):
    """The replicas' contexts: cell scan (with or without the row pass), or the
    constraint graph (graph=True; cells then only set the graph's build)."""
    return [ecmc.System(r.start.x, r.start.y, r.start.active, r.start.box, r.ell,
                        cells_per_side=cells_for(r.start, cells), undo_cap=undo_cap,
                        stream=stream, rowpass=rowpass, graph=graph) for r in reps]


# parallel pass of a trial: the row pass (cell scan), the general pass (cell
# scan), or the constraint graph
SEARCHES = {"row": dict(rowpass=True, graph=False), "general": dict(rowpass=False, graph=False),
            "graph": dict(rowpass=False, graph=True)}
# chains a warp advances in each search: one (the warp's lanes share a chain's
# scan) or 32 (graph mode: a chain per thread)
CHAINS_PER_WARP = {"row": 1, "general": 1, "graph": 32}


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


def run_plain(systems, budget: int, legs_per_launch: int = 1 << 20):
    """One system at a time through ecmc_run_to_breakpoint, each in as few
    launches as the budget allows (the budget stops a launch at the first
    breakpoint where it is met)."""
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


def _hardware_key() -> str:
    """The GPU and the build of the library: a cached choice holds for both."""
    try:
        import torch
        gpu = torch.cuda.get_device_name(0).replace(" ", "_")
    except Exception:  # pragma: no cover
        gpu = "unknown"
    try:
        import hashlib
        with open(ecmc.library_path(), "rb") as f:
            lib = hashlib.sha256(f.read()).hexdigest()[:16]
    except Exception:
        lib = "unknown"
    return f"{gpu}_{lib}"


def _key(reps: list[Replica]) -> str:
    ns = sorted(r.start.n for r in reps)
    return f"{_hardware_key()}_n{ns[0]}-{ns[-1]}_r{len(reps)}"


def autotune(reps: list[Replica], trial_budget: int = 20_000,
             cells_options=("lattice", "default"), search_options=("row", "general", "graph"),
             legs_options=(4, 16, 64), cache: str | None = CACHE, stream=None) -> dict:
    """Tries every (cell size, parallel pass, legs per launch) on a sample of
    the replicas and keeps the fastest by liftings per device second; every
    trial is recorded, and the choice is cached per GPU, library build and
    workload. The parallel pass is the row pass (a warp holds 32 slots of
    its chain's row and runs prepared steps in batches), the general pass (a
    warp scans 3 rows x 2 columns of cells per pass), both one chain per
    warp, or the constraint graph (one chain per thread; its cell size only
    sets the graph's build, so it is tried once). Fewer warps per chain (two
    chains per warp) are not offered: every FP64 warp instruction occupies
    the sub-partition's FP64 unit ~64 cycles whatever its lane mask, so a
    warp's latency per step is set by its FP64 instruction count, which two
    chains would not share."""
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
    combos = [(cells, search) for search in search_options for cells in cells_options
              if search != "graph" or cells == cells_options[0]]
    for cells, search in combos:
        systems = create(sample, cells, stream=stream, **SEARCHES[search])
        try:
            for legs in legs_options:
                lifts, ms, _ = run_batched(systems, trial_budget, legs, stream=stream)
                rate = lifts / (ms / 1e3) if ms > 0 else 0.0
                rows = sum(q.stats()["row_windows"] for q in systems)
                trials.append({"cells": cells, "search": search, "legs_per_launch": legs,
                               "chains_per_warp": CHAINS_PER_WARP[search],
                               "liftings_per_s": rate, "row_windows": rows})
                if best is None or rate > best["liftings_per_s"]:
                    best = dict(trials[-1])
        finally:
            for q in systems:
                q.close()
    best["trials"] = trials
    best["key"] = key
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


def bench_batched(count: int = 512, budget: int = 1_000_000, same_budget: int = 50_000,
                  seed: int = 0, tune: bool = True, stream=None, cache: str | None = CACHE) -> dict:
    """Batched throughput of `count` replicas to `budget` liftings each; and,
    on the same replicas with `same_budget` liftings each, batched against one
    at a time (both rates over the same systems and the same work)."""
    reps = make_replicas(count, seed)
    choice = autotune(reps, stream=stream, cache=cache) if tune else {
        "cells": "lattice", "search": "row", "legs_per_launch": 16}
    cells, legs = choice["cells"], choice["legs_per_launch"]
    mode = SEARCHES[choice["search"]]
    t0 = time.perf_counter()
    systems = create(reps, cells, stream=stream, **mode)
    t_create = time.perf_counter() - t0
    try:
        lifts, ms, launches = run_batched(systems, budget, legs, stream)
    finally:
        for q in systems:
            q.close()
    systems = create(reps, cells, stream=stream, **mode)
    try:
        s_lifts, s_ms, _ = run_batched(systems, same_budget, legs, stream)
    finally:
        for q in systems:
            q.close()
    systems = create(reps, cells, stream=stream, **mode)
    try:
        p_lifts, p_ms, p_launches = run_plain(systems, same_budget)
    finally:
        for q in systems:
            q.close()
    same = s_lifts / (s_ms / 1e3)
    plain = p_lifts / (p_ms / 1e3)
    return {"replicas": count, "budget_per_replica": budget, "liftings": lifts,
            "device_ms": ms, "launches": launches, "liftings_per_s": lifts / (ms / 1e3),
            "create_s": t_create,
            "same_set": {"budget_per_replica": same_budget, "batched_liftings_per_s": same,
                         "one_at_a_time_liftings_per_s": plain,
                         "one_at_a_time_launches": p_launches,
                         "batched_over_one_at_a_time": same / plain if plain else None},
            "autotune": {k: v for k, v in choice.items() if k != "trials"},
            "autotune_trials": choice.get("trials")}
