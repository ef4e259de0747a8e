"""Benchmark: ECMC liftings per second on one GB300 (N = 2^20 disks, eta = 0.72).

Workload: a 1024 x 1024 jittered square lattice (seeded), eta = 0.72, k
chains (default 1024), chain length ell = 1 between breakpoints, v = +x.
One step = one ecmc_run_to_breakpoint call of --legs legs. ``value`` is
liftings per second of device time (CUDA events on the context's stream,
inputs resident in HBM), ``e2e`` the same metric through the C-ABI with host
buffers (create from host x/y, run, read positions back) inside the timed
region. The working set (~100 MB) is below the 129 MB L2, so L2 is flushed
with a 512 MB write between timed steps.

The default run (--search cells: the cell scan, one warp per chain) also
measures the same workload in constraint-graph mode (ECMC_GRAPH: liftings
through the arrows of G(3), Sec. 3.1) and adds it as "graph_mode" with its own
roofline and e2e numbers; --search graph makes graph mode the headline.

--impl reference times the CPU oracle (plain C, one core) on a bounded
sample of the same workload.

--workload batched: many independent replicas of uneven size (N log-uniform
in [1024, 65536], eta uniform in [0.60, 0.74], k = sqrt(N), a liftings budget
each) advanced by one persistent launch per slice, against the same systems
one at a time. --workload serve: a seeded Poisson stream of whole-ECMC
requests through the continuous-batching server (p50/p99 latency).
--workload conflicts: the conflict (violation) rate per leg against the
number of chains, n / sqrt(N): N = 128^2 at eta = 0.708 with 128 chains, and
N = 2^20 at eta = 0.72 with 256 ... 16384 chains, each run to --target
liftings; cell claims with one window per leg (the leg-level flag) and with
several windows (per-window flags), and graph mode with one window (the flag
from the disks that isolated chains read).

Multi-GPU: the path does not shard a single system; every rank runs an
independent replica (its own seed), ``value`` sums all ranks' liftings over
the slowest rank's time ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_LIFTING = 104  # algorithmic: read x,y,t of <= 3 neighbours (72 B), write x_i,t_i,t_j + 2 tags (32 B)
METRIC = "liftings/s (ECMC events/s), N=2^20 hard disks, eta=0.72, ell=1"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--k", type=int, default=1024, help="chains")
    p.add_argument("--legs", type=int, default=10, help="legs per step")
    p.add_argument("--search", default="cells", choices=["cells", "graph"],
                   help="lifting search of the headline: cell scan (default) or the "
                        "constraint graph G(3); the default run measures graph mode too")
    p.add_argument("--restart", action="store_true",
                   help="graph mode: conflicts by restart strategy 2 (Sec. 3.4) instead of "
                        "the local repair")
    p.add_argument("--windows", type=int, default=0,
                   help="claim windows per leg (0: cell scan 1 up to 1024 chains, 2 up to 4096, "
                        "else 4; graph 1)")
    p.add_argument("--workload", default="lattice",
                   choices=["lattice", "batched", "serve", "conflicts"])
    p.add_argument("--target", type=float, default=1e9,
                   help="liftings per point (conflicts workload)")
    p.add_argument("--replicas", type=int, default=512)
    p.add_argument("--budget", type=float, default=1e6, help="liftings per replica (batched)")
    p.add_argument("--requests", type=int, default=200)
    p.add_argument("--rate", type=float, default=50.0, help="request arrivals per second")
    p.add_argument("--m", type=int, default=1024, help="lattice side (N = m*m)")
    p.add_argument("--eta", type=float, default=0.72)
    p.add_argument("--ell", type=float, default=1.0)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    a = p.parse_args()
    a.windows_arg = a.windows
    a.windows = windows_for(a, a.search)
    return a


def windows_for(a, search):
    """Claim windows per leg: as given, else the measured best of each search."""
    if a.windows_arg > 0:
        return a.windows_arg
    if search == "graph":
        return 1
    # measured (N = 2^20 lattices, W in 1, 2, 4): one window up to k = 4096,
    # two at k = 16384
    return 1 if a.k <= 4096 else 2


def workload(a, search=None):
    search = search or a.search
    return {"workload": f"lattice {a.m}x{a.m} (N={a.m * a.m}) eta={a.eta} jitter=0.01, "
                        f"k={a.k} chains, ell={a.ell}, v=+x, {a.legs} legs/step",
            "n": a.m * a.m, "eta": a.eta, "k": a.k, "ell": a.ell, "legs_per_step": a.legs,
            "search": "cell scan" if search == "cells" else (
                "constraint graph G(3), restart strategy 2" if a.restart
                else "constraint graph G(3)"),
            "claim_windows_per_leg": windows_for(a, search),
            "seed": a.seed, "l2": "flushed between steps (512 MB write)"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for s in self.samples for q in range(4)
                          if len(s) > 4 + q and s[4 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------- helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source file is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        k = d.get("kernels", {}).get(kernel, {})
        src = open(os.path.join(ROOT, "paper_2004_11040_gb300", "csrc", k["source"]), "rb").read()
        if k.get("source_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return k.get("dram_bytes_per_launch")
    except Exception:
        return None


def cpu_baseline(a, start, budget_s):
    """The oracle as it stands, one host core, on whole legs of the same workload."""
    from oracle import oracle as O
    O.build()
    x, act = start.x.copy(), start.active.copy()
    lifts, legs = 0, 0
    t0 = time.perf_counter()
    while True:
        r = O.run_leg(x, start.y, act, start.box, a.ell, log=False)
        x, act = r.x, r.active
        lifts += r.lifts
        legs += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": lifts / el, "unit": "liftings/s", "cores": 1, "kind": "oracle",
            "sample": f"{legs} whole legs ({lifts} liftings) of the same workload in {el:.1f} s"}


def cpu_multicore(a, start, budget_s):
    """The paper's Alg. 5 (OpenMP threads, atomic CAS on tags) on all host
    cores, whole legs of the same workload; horizon violations are counted,
    not repaired (the paper's benchmark mode)."""
    from oracle import alg5
    first = alg5.run(start.x, start.y, start.active, start.box, a.ell, 1)
    legs = max(1, int(budget_s / max(first.seconds, 1e-3)))
    r = alg5.run(start.x, start.y, start.active, start.box, a.ell, legs)
    return {"value": r.lifts / r.seconds, "unit": "liftings/s", "cores": r.threads,
            "kind": "paper Alg. 5 on host threads (OpenMP, atomic CAS on tags)",
            "sample": f"{legs} whole legs ({r.lifts} liftings) of the same workload in "
                      f"{r.seconds:.1f} s; {r.violations} horizon violations counted, "
                      f"not repaired"}


def host_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def aggregate(dev_ms, lifts, ws, device="cpu"):
    """Whole-job numbers of a replicas-only run: the slowest rank's time and
    all ranks' liftings (a rank that exits early simply contributes nothing
    beyond its own count). With ws == 1 the rank's own numbers."""
    if ws <= 1:
        return dev_ms, lifts
    import torch
    import torch.distributed as dist
    tt = torch.tensor([dev_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ll = torch.tensor([float(lifts)], device=device, dtype=torch.float64)
    dist.all_reduce(ll, op=dist.ReduceOp.SUM)
    return float(tt.item()), int(ll.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ reference

def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2004_11040_gb300 import synth
    start = synth.lattice_start(a.m, a.eta, a.k, seed=a.seed)
    budget = max(2.0, 60.0 / max(1, a.steps + a.warmup))
    cb = None
    vals = []
    for s in range(a.warmup + a.steps):
        r = cpu_baseline(a, start, budget)
        if s >= a.warmup:
            vals.append(r["value"])
            cb = r
    v = sum(vals) / len(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "liftings/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1000.0 * budget, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(a),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "liftings/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours

def measure(a, search, start, stream, flush, barrier, ws):
    """Times --steps steps of one search mode (after --warmup steps) and the
    end-to-end C-ABI path; returns the numbers of one JSON line."""
    import numpy as np
    import torch

    from paper_2004_11040_gb300 import ecmc
    graph = search == "graph"
    W = windows_for(a, search)
    sysm = ecmc.System(start.x, start.y, start.active, start.box, a.ell, stream=stream,
                       windows=W, graph=graph, restart=graph and a.restart)
    for _ in range(a.warmup):
        sysm.run(a.legs)
    st0, pr0 = sysm.stats(), sysm.profile()
    dev_ms = 0.0
    lifts = 0
    barrier()
    for _ in range(a.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        b = sysm.stats()
        sysm.run(a.legs)
        e = sysm.stats()
        dev_ms += e["device_ms"] - b["device_ms"]
        lifts += e["liftings"] - b["liftings"]
    barrier()
    st1, pr1 = sysm.stats(), sysm.profile()
    t_max, tot_lifts = aggregate(dev_ms, lifts, ws, device="cuda")
    # the hot path is one persistent kernel launch per step
    kname = "k_run_graph" if graph else "k_run"
    kms = dev_ms / a.steps  # CUDA events around each launch, on its stream
    kl = lifts / a.steps
    peak, peak_kind = peaks()
    achieved = (kl * BYTES_PER_LIFTING) / (kms / 1000.0) / 1e9 if kms > 0 else 0.0

    # end to end through the C-ABI with host buffers
    nx = start.n
    e2e_lifts, e2e_s = 0, 0.0
    h2d = 2 * nx * 8 + 4 * a.k
    d2h = 2 * nx * 8 + 4 * a.k
    hx = torch.from_numpy(start.x).pin_memory().numpy()
    hy = torch.from_numpy(start.y).pin_memory().numpy()
    ha = torch.from_numpy(start.active.astype(np.int32)).pin_memory().numpy()
    ox = torch.empty(nx, dtype=torch.float64).pin_memory().numpy()
    ot = torch.empty(nx, dtype=torch.float64).pin_memory().numpy()
    oa = torch.empty(a.k, dtype=torch.int32).pin_memory().numpy()
    for s in range(max(1, a.steps // 2) + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = ecmc.ecmc_create(sysm.params, hx, hy, ha, stream)
        fl = np.zeros(a.legs, dtype=np.uint8)
        ecmc.ecmc_run_to_breakpoint(ctx, a.legs, 0, fl)
        ecmc.ecmc_positions(ctx, ox, None, ot, oa)
        el = time.perf_counter() - t0
        n_l = ecmc.ecmc_stats(ctx)["liftings"]
        ecmc.ecmc_destroy(ctx)
        if s > 0:
            e2e_lifts += n_l
            e2e_s += el
    sysm.close()
    return {
        "value": tot_lifts / (t_max / 1000.0), "t_max": t_max, "liftings": tot_lifts,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_for(kname), "kernel": kname,
                     "peak_source": peak_kind, "bytes_per_lifting": BYTES_PER_LIFTING,
                     "kernel_ms_per_launch": kms, "liftings_per_launch": kl},
        "e2e": {"value": e2e_lifts / e2e_s, "unit": "liftings/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": a.steps,
        "detail": {"legs": st1["legs"] - st0["legs"],
                   "conflict_legs": st1["conflict_legs"] - st0["conflict_legs"],
                   "repaired_chains": st1["repaired_chains"] - st0["repaired_chains"],
                   "continued_chains": st1["continued_chains"] - st0["continued_chains"],
                   "restarts": st1["restarts"] - st0["restarts"],
                   "liftings": tot_lifts,
                   "profile": {key: pr1[key] - pr0[key] for key in pr1},
                   "horizon_asserts": st1["horizon_asserts"],
                   "order_errors": st1["order_errors"]},
    }


def run_ours(a):
    import torch

    from paper_2004_11040_gb300 import build, synth
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    start = synth.lattice_start(a.m, a.eta, a.k, seed=a.seed + rank)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        head = measure(a, a.search, start, stream, flush, barrier, ws)
    other = None
    if a.search == "cells":
        # the constraint-graph mode on the same workload (same Alg. 2 results)
        other = measure(a, "graph", start, stream, flush, barrier, ws)

    if rank != 0:
        return
    cb = cbm = None
    if ws == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(a, start, a.cpu_seconds)
        cbm = cpu_multicore(a, start, a.cpu_seconds / 2)
    line = {
        "metric": METRIC, "value": head["value"], "unit": "liftings/s", "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": head["t_max"] / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload(a),
        "roofline": head["roofline"],
        "cpu_baseline": cb, "cpu_baseline_multicore": cbm, "host": host_info(),
        "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
        "clocks": clk.summary(),
        "detail": head["detail"],
    }
    if other is not None:
        line["graph_mode"] = {
            "value": other["value"], "unit": "liftings/s",
            "ms_per_step": other["t_max"] / a.steps, "config": workload(a, "graph"),
            "roofline": other["roofline"], "e2e": other["e2e"],
            "gpu_launches": other["gpu_launches"], "detail": other["detail"]}
    print(json.dumps(line), flush=True)


# ------------------------------------------------- batched replicas / serving

def run_batched_bench(a):
    """Replicas of uneven size to a liftings budget each: one persistent launch
    per slice for all of them, against the same systems one at a time."""
    import torch

    from paper_2004_11040_gb300 import batch, build
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    reps = batch.make_replicas(a.replicas, seed=a.seed + rank)
    choice = batch.autotune(reps, stream=stream, cache=None)
    systems = batch.create(reps, choice["cell_factor"], stream=stream)
    try:
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            lifts, ms, launches = batch.run_batched(systems, int(a.budget),
                                                    choice["legs_per_launch"], stream)
            wall = time.perf_counter() - t0
    finally:
        for q in systems:
            q.close()
    sample = min(16, len(reps))
    plain = batch.create(reps[:sample], choice["cell_factor"], stream=stream)
    try:
        p_lifts, p_ms, p_launches = batch.run_plain(plain, int(a.budget), choice["legs_per_launch"])
    finally:
        for q in plain:
            q.close()
    if rank != 0:
        return
    v, pv = lifts / (ms / 1e3), p_lifts / (p_ms / 1e3)
    print(json.dumps({
        "metric": "batched liftings/s over all replicas", "value": v, "unit": "liftings/s",
        "n_gpus": ws, "steps": launches, "warmup": 0, "ms_per_step": ms / max(1, launches),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{a.replicas} replicas, N log-uniform [1024, 65536] (lattice), "
                               f"eta U[0.60, 0.74], k = sqrt(N), ell = 1, "
                               f"{int(a.budget)} liftings each", "seed": a.seed},
        "wall_liftings_per_s": lifts / wall, "autotune": {k: v2 for k, v2 in choice.items()
                                                          if k != "trials"},
        "one_at_a_time": {"value": pv, "unit": "liftings/s", "sample_replicas": sample,
                          "launches": p_launches},
        "batched_over_one_at_a_time": v / pv, "gpu_launches": launches,
        "clocks": clk.summary()}), flush=True)


def run_serve_bench(a):
    """A seeded Poisson stream of whole-ECMC requests through the server."""
    import torch

    from paper_2004_11040_gb300 import build, serve
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    reqs = serve.make_requests(a.requests, seed=a.seed + rank, rate=a.rate,
                               budget_range=(1e4, max(1e4, a.budget)))
    serve.prepare(reqs)
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(hbm_budget_bytes=int(free * 0.6), stream=stream)
    try:
        with ClockSampler(local) as clk:
            st = srv.serve(reqs)
    finally:
        srv.close()
    # the same requests one at a time (a sample), device time
    sample = reqs[: min(12, len(reqs))]
    one_lifts, one_ms = 0, 0.0
    for r in sample:
        from paper_2004_11040_gb300 import ecmc
        q = r.start
        sysm = ecmc.System(q.x, q.y, q.active, q.box, 1.0, undo_cap=srv.undo_cap, stream=stream)
        got = 0
        while got < r.budget:
            b = sysm.stats()
            sysm.run(srv.slice_legs, event_budget=r.budget - got)
            e = sysm.stats()
            got += e["liftings"] - b["liftings"]
            one_ms += e["device_ms"] - b["device_ms"]
        one_lifts += got
        sysm.close()
    if rank != 0:
        return
    summ = st.summary()
    one = one_lifts / (one_ms / 1e3)
    print(json.dumps({
        "metric": "served liftings/s (device) with p50/p99 request latency",
        "value": summ["liftings_per_s_device"], "unit": "liftings/s", "n_gpus": ws,
        "steps": summ["slices"], "warmup": 0,
        "ms_per_step": summ["device_ms"] / max(1, summ["slices"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{a.requests} requests, Poisson {a.rate}/s, N log-uniform "
                               f"[4096, 4194304] (lattice), eta U[0.62, 0.72], k = sqrt(N), "
                               f"budget log-uniform [1e4, {a.budget:g}] liftings",
                   "seed": a.seed},
        "serve": summ,
        "one_at_a_time": {"value": one, "unit": "liftings/s", "sample_requests": len(sample)},
        "served_over_one_at_a_time": summ["liftings_per_s_device"] / one if one else None,
        "clocks": clk.summary()}), flush=True)


def run_conflicts(a):
    """Conflict rate per leg and the fraction of chains repaired, against
    n / sqrt(N). The flag: the cells (cell scan) or the disks (graph mode) that
    isolated chains read overlap."""
    import torch

    from paper_2004_11040_gb300 import build, ecmc, synth
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    stream = torch.cuda.current_stream()
    points = [(128, 0.708, 128), (1024, 0.72, 256), (1024, 0.72, 1024), (1024, 0.72, 4096),
              (1024, 0.72, 16384)]
    out = []
    # (search, windows): cell claims with one and with several windows; graph
    # mode (flag = overlap of the disks isolated chains read) with one window.
    # --search graph: the graph-mode points alone
    for m, eta, k in points:
        start = synth.lattice_start(m, eta, k, seed=a.seed)
        modes = [("cells", 1), ("cells", 2 if k <= 4096 else 4), ("graph", 1)]
        if a.search == "graph":
            modes = modes[2:]
        for search, windows in modes:
            graph = search == "graph"
            sysm = ecmc.System(start.x, start.y, start.active, start.box, 1.0, stream=stream,
                               windows=windows, graph=graph)
            # the one-window cell runs of many chains repair for long: bounded sample
            target = a.target if graph or windows > 1 or k <= 1024 else min(a.target, 2e7)
            flags = []
            t0 = time.perf_counter()
            while sysm.stats()["liftings"] < target:
                f, _ = sysm.run(50)
                flags.extend(int(v) for v in f)
            st = sysm.stats()
            sysm.close()
            legs = st["legs"]
            out.append({"N": m * m, "eta": eta, "k": k, "n_over_sqrtN": k / m,
                        "search": search, "claim_windows": windows, "legs": legs, "liftings": st["liftings"],
                        "conflict_rate_per_leg": st["conflict_legs"] / legs,
                        "repaired_chains_per_leg_per_chain": st["repaired_chains"] / legs / k,
                        "liftings_per_s": st["liftings"] / (st["device_ms"] / 1e3),
                        "horizon_asserts": st["horizon_asserts"],
                        "order_errors": st["order_errors"],
                        "wall_s": time.perf_counter() - t0})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "conflict rate per leg vs n/sqrt(N)", "unit": "fraction",
                      "n_gpus": 1, "data": "synthetic", "dtype": "f64",
                      "config": {"workload": "jittered square lattices, ell = 1, v = +x",
                                 "target_liftings_per_point": a.target, "seed": a.seed},
                      "points": out}), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched_bench(args)
    elif args.workload == "serve":
        run_serve_bench(args)
    elif args.workload == "conflicts":
        run_conflicts(args)
    else:
        run_ours(args)
