"""Benchmark: ECMC liftings per second on one GB300 (N = 2^20 disks, eta = 0.72).

Headline workload (the metric's configuration): a 1024 x 1024 jittered square
lattice (seeded), eta = 0.72, k = 1024 chains, chain length ell = 1 between
breakpoints, v = +x, on cells aligned with the start lattice (one cell per
lattice site: every row of disks lies inside one cell row, rows out of reach
of each other, so the row pass applies). One step = one
ecmc_run_to_breakpoint call of --legs legs. ``value`` is liftings per second
of device time (CUDA events on the context's stream, inputs resident in HBM);
``e2e`` the same metric through the C-ABI with host buffers (create from host
x/y, run, read positions back) inside the timed region. The state (~150 MB)
is close to the 129 MB L2, so L2 is flushed with a 512 MB write between timed
steps.

The default run also measures, each with the same timing rules:
  graph_mode      the headline workload in constraint-graph mode (ECMC_GRAPH,
                  Sec. 3.1), with its own roofline and e2e;
  config3_sweep   k in {256, 1024, 4096, 16384} chains (n / sqrt(N) = 1/4 ..
                  16), W = 1: liftings/s, roofline, conflict rates;
  batched         512 replicas (N log-uniform in [1024, 65536], eta uniform
                  in [0.60, 0.74], k = sqrt(N)) to 10^6 liftings each in
                  persistent launches over all of them; and, on the same 512
                  replicas with a smaller budget each, batched against one at
                  a time (same systems, same work);
  served          a seeded Poisson stream of whole-ECMC requests through the
                  continuous-batching server (p50/p99 latency), against the
                  same requests one at a time (a sample stratified over N);
  cpu_baseline    the oracle on one host core (a bounded sample of legs), and
                  cpu_baseline_multicore: the paper's Alg. 5 on all host cores.
--quick skips the sweep, the batched and the served records.

--impl reference times the CPU oracle (plain C, one core) on a bounded
sample of the same workload.

--workload batched | serve | conflicts: one of those measurements alone
(conflicts: the conflict rate per leg against n / sqrt(N), configs 2 and 3).

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
    p.add_argument("--cells", default="lattice", choices=["lattice", "default"],
                   help="cell grid: one cell per start-lattice site (default), or the "
                        "library's smallest cells of side >= d")
    p.add_argument("--restart", action="store_true",
                   help="graph mode: conflicts by restart strategy 2 (Sec. 3.4) instead of "
                        "the local repair")
    p.add_argument("--windows", type=int, default=0,
                   help="claim windows per leg (0: one window, the measured best)")
    p.add_argument("--workload", default="lattice",
                   choices=["lattice", "batched", "serve", "conflicts"])
    p.add_argument("--quick", action="store_true",
                   help="headline, graph mode and CPU baselines only")
    p.add_argument("--target", type=float, default=5e7,
                   help="liftings per point (conflicts workload)")
    p.add_argument("--replicas", type=int, default=512)
    p.add_argument("--budget", type=float, default=1e6, help="liftings per replica (batched)")
    p.add_argument("--same-budget", type=float, default=1e5,
                   help="liftings per replica of the batched vs one-at-a-time comparison")
    p.add_argument("--requests", type=int, default=1000)
    p.add_argument("--rate", type=float, default=0.0,
                   help="request arrivals per second (0: 80%% of the device's capacity, "
                        "taken as the batched liftings/s over the mean budget)")
    p.add_argument("--serve-budget", type=float, nargs=2, default=(1e5, 1e8),
                   help="request budget range, liftings (log-uniform)")
    p.add_argument("--m", type=int, default=1024, help="lattice side (N = m*m)")
    p.add_argument("--eta", type=float, default=0.72)
    p.add_argument("--ell", type=float, default=1.0)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


SWEEP_K = (256, 1024, 4096, 16384)


def windows_for(a, search, k=None):
    """Claim windows per leg: as given, else the measured best of each search."""
    k = a.k if k is None else k
    if a.windows > 0:
        return a.windows
    # measured on N = 2^20 lattices (W in 1, 2, 16, 64): one window per leg is the
    # fastest at every k in both searches
    return 1


def cells_of(a):
    """Cells per side of the headline: one per lattice site, or 0 (default)."""
    return a.m if a.cells == "lattice" else 0


def workload(a, search=None, k=None):
    search = search or a.search
    k = a.k if k is None else k
    return {"workload": f"lattice {a.m}x{a.m} (N={a.m * a.m}) eta={a.eta} jitter=0.01, "
                        f"k={k} chains, ell={a.ell}, v=+x, {a.legs} legs/step",
            "n": a.m * a.m, "eta": a.eta, "k": k, "ell": a.ell, "legs_per_step": a.legs,
            "search": "cell scan" if search == "cells" else (
                "constraint graph G(3), restart strategy 2" if a.restart
                else "constraint graph G(3)"),
            "cells_per_side": cells_of(a) or "library default (side >= d)",
            "claim_windows_per_leg": windows_for(a, search, k),
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
    """DRAM bytes per lifting of `kernel` from the committed ncu summary, if the
    kernel's source files are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        k = d.get("kernels", {}).get(kernel, {})
        h = hashlib.sha256()
        for name in k["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2004_11040_gb300", "csrc", name), "rb").read())
        if k.get("sources_sha256") != h.hexdigest():
            return None
        return k.get("dram_bytes_per_lifting")
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

def measure(a, search, start, stream, flush, barrier, ws, nc, e2e=True):
    """Times --steps steps of one search mode (after --warmup steps) and, with
    e2e, the end-to-end C-ABI path; returns the numbers of one record."""
    import numpy as np
    import torch

    from paper_2004_11040_gb300 import ecmc
    graph = search == "graph"
    k = start.k
    W = windows_for(a, search, k)
    sysm = ecmc.System(start.x, start.y, start.active, start.box, a.ell, stream=stream,
                       windows=W, graph=graph, restart=graph and a.restart, cells_per_side=nc)
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
    # the hot path is one persistent kernel launch per step, timed by CUDA
    # events around the launch on the context's stream
    kname = "k_run_graph" if graph else "k_run"
    kms = dev_ms / a.steps
    kl = lifts / a.steps
    peak, peak_kind = peaks()
    achieved = (kl * BYTES_PER_LIFTING) / (kms / 1000.0) / 1e9 if kms > 0 else 0.0
    per_lift = traffic_for(kname)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": per_lift * kl if per_lift else None, "kernel": kname,
            "bytes_per_lifting": BYTES_PER_LIFTING, "kernel_ms_per_launch": kms,
            "liftings_per_launch": kl}
    if per_lift:
        # the same launch against the DRAM bytes ncu counted per lifting
        dram = per_lift * kl / (kms / 1000.0) / 1e9
        roof["dram_bytes_per_lifting"] = per_lift
        roof["dram_achieved"] = dram
        roof["dram_frac"] = dram / peak

    legs = st1["legs"] - st0["legs"]
    d = {key: st1[key] - st0[key] for key in ("legs", "conflict_legs", "conflict_windows",
                                               "blocked_chains", "repaired_chains",
                                               "continued_chains", "restarts", "row_windows")}
    windows = legs * W
    detail = dict(d)
    detail.update({
        "liftings": tot_lifts,
        "claim_windows": windows,
        "conflict_windows_per_window": d["conflict_windows"] / windows if windows else None,
        "met_chains_per_window_per_chain": d["blocked_chains"] / windows / k if windows else None,
        "repaired_chains_per_leg_per_chain": d["repaired_chains"] / legs / k if legs else None,
        "row_pass_windows_fraction": d["row_windows"] / windows if windows else None,
        "us_per_leg": 1000.0 * dev_ms / legs if legs else None,
        "liftings_per_chain_per_leg": lifts / legs / k if legs else None,
        "profile": {key: pr1[key] - pr0[key] for key in pr1},
        "horizon_asserts": st1["horizon_asserts"], "order_errors": st1["order_errors"],
        "device_bytes": st1["device_bytes"]})

    out = {"value": tot_lifts / (t_max / 1000.0), "t_max": t_max, "liftings": tot_lifts,
           "roofline": roof, "gpu_launches": a.steps, "detail": detail,
           "claim_windows_per_leg": W}
    if e2e:
        # end to end through the C-ABI with host buffers: create from pinned
        # host x, y, active; run one step; read x, t, active back
        nx = start.n
        e2e_lifts, e2e_s = 0, 0.0
        # (bytes of the whole job's step: every rank copies its own system)
        h2d = ws * (2 * nx * 8 + 4 * k)
        d2h = ws * (2 * nx * 8 + 4 * k)
        hx = torch.from_numpy(start.x).pin_memory().numpy()
        hy = torch.from_numpy(start.y).pin_memory().numpy()
        ha = torch.from_numpy(start.active.astype(np.int32)).pin_memory().numpy()
        ox = torch.empty(nx, dtype=torch.float64).pin_memory().numpy()
        ot = torch.empty(nx, dtype=torch.float64).pin_memory().numpy()
        oa = torch.empty(k, dtype=torch.int32).pin_memory().numpy()
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
        # whole job over the ranks, as the device value: all ranks' liftings
        # over the slowest rank's time (the rank's own with one GPU)
        e2e_ms, e2e_lifts = aggregate(e2e_s * 1000.0, e2e_lifts, ws, device="cuda")
        e2e_s = e2e_ms / 1000.0
        out["e2e"] = {"value": e2e_lifts / e2e_s, "unit": "liftings/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "includes": "context creation from host positions (cell build), "
                                  f"{a.legs} legs, positions/times/active read back"}
        out["gpu_launches_e2e_step"] = 1
    sysm.close()
    return out


def sweep(a, stream, flush, barrier, ws, rank, head, clk_index):
    """Config 3: k chains in {256, 1024, 4096, 16384} on the same N and eta,
    in both searches; per point liftings/s, roofline, W and conflict rates
    (the Sec. 3.4 birthday scaling against k^2 / N)."""
    from paper_2004_11040_gb300 import synth
    out = []
    n = a.m * a.m
    for k in SWEEP_K:
        start = synth.lattice_start(a.m, a.eta, k, seed=a.seed + rank)
        for search in ("cells", "graph"):
            if head and k == a.k and search in head:
                r = head[search]
            else:
                with ClockSampler(clk_index) as clk:
                    r = measure(a, search, start, stream, flush, barrier, ws, cells_of(a),
                                e2e=False)
                r["clocks"] = clk.summary()
            dt = r["detail"]
            out.append({"k": k, "n_over_sqrtN": k / a.m, "k2_over_N": k * k / n,
                        "search": search, "claim_windows_per_leg": r["claim_windows_per_leg"],
                        "value": r["value"], "unit": "liftings/s",
                        "ms_per_step": r["t_max"] / a.steps,
                        "roofline": {q: r["roofline"][q] for q in
                                     ("achieved", "peak", "frac", "traffic", "unit")},
                        "conflict_legs_per_leg": dt["conflict_legs"] / dt["legs"],
                        "conflict_windows_per_window": dt["conflict_windows_per_window"],
                        "met_chains_per_window_per_chain": dt["met_chains_per_window_per_chain"],
                        "repaired_chains_per_leg_per_chain":
                            dt["repaired_chains_per_leg_per_chain"],
                        "row_pass_windows_fraction": dt["row_pass_windows_fraction"],
                        "us_per_leg": dt["us_per_leg"],
                        "clocks": r.get("clocks")})
    return out


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

    t_begin = time.perf_counter()
    with ClockSampler(local) as clk:
        head = measure(a, a.search, start, stream, flush, barrier, ws, cells_of(a))
    other_search = "graph" if a.search == "cells" else "cells"
    with ClockSampler(local) as clk2:
        other = measure(a, other_search, start, stream, flush, barrier, ws, cells_of(a))
    other["clocks"] = clk2.summary()
    del start
    extra = {}
    if not a.quick:
        extra["config3_sweep"] = sweep(a, stream, flush, barrier, ws, rank,
                                       {a.search: head, other_search: other}, local)
        del flush
        torch.cuda.empty_cache()
        if ws == 1:
            extra["batched"] = batched_record(a, stream, local)
            extra["served"] = served_record(a, stream, local,
                                            capacity=extra["batched"]["value"])
    if rank != 0:
        return
    cb = cbm = None
    if ws == 1 and not a.no_cpu_baseline:
        cstart = synth.lattice_start(a.m, a.eta, a.k, seed=a.seed)
        cb = cpu_baseline(a, cstart, a.cpu_seconds)
        cbm = cpu_multicore(a, cstart, a.cpu_seconds / 2)
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
    if cb:
        line["ratios"] = {"value_over_cpu_oracle": head["value"] / cb["value"],
                          "value_over_cpu_multicore": head["value"] / cbm["value"],
                          "e2e_over_cpu_multicore": head["e2e"]["value"] / cbm["value"]}
    key = "graph_mode" if other_search == "graph" else "cell_mode"
    line[key] = {
        "value": other["value"], "unit": "liftings/s",
        "ms_per_step": other["t_max"] / a.steps, "config": workload(a, other_search),
        "roofline": other["roofline"], "e2e": other["e2e"],
        "gpu_launches": other["gpu_launches"], "detail": other["detail"],
        "clocks": other["clocks"]}
    line.update(extra)
    line["wall_s"] = time.perf_counter() - t_begin
    print(json.dumps(line), flush=True)


# ------------------------------------------------- batched replicas / serving

def batched_record(a, stream, clk_index):
    """Config 4: 512 replicas of uneven size, each to --budget liftings, in
    persistent launches over all of them (the autotuner's choice of cells,
    parallel pass and legs per launch); and the same replicas with
    --same-budget liftings each, batched against one at a time."""
    from paper_2004_11040_gb300 import batch
    with ClockSampler(clk_index) as clk:
        r = batch.bench_batched(a.replicas, int(a.budget), int(a.same_budget), seed=a.seed,
                                stream=stream, cache=None)
    r["clocks"] = clk.summary()
    r["config"] = {"workload": f"{a.replicas} replicas, N log-uniform [1024, 65536] (lattice), "
                               f"eta U[0.60, 0.74], k = sqrt(N), ell = 1, "
                               f"{int(a.budget)} liftings each; batched vs one at a time on "
                               f"the same {a.replicas} replicas, {int(a.same_budget)} "
                               f"liftings each", "seed": a.seed}
    r["value"] = r["liftings_per_s"]
    r["unit"] = "liftings/s"
    return r


def served_record(a, stream, clk_index, capacity=None):
    """Config 5 (a bounded sample): a seeded Poisson stream of whole-ECMC
    requests through the continuous-batching server, p50/p99 latency; and the
    same requests one at a time (a sample stratified over N). The arrival
    rate aims at 80% occupancy: 0.8 x capacity / mean budget, the capacity
    being the batched liftings/s measured before (else --rate)."""
    import numpy as np
    import torch

    from paper_2004_11040_gb300 import serve
    mean_budget = serve.Server.mean_budget(a.serve_budget)
    if a.rate > 0 or not capacity:
        rate, rate_from = (a.rate or 20.0), "given"
    else:
        rate = 0.8 * capacity / mean_budget
        rate_from = (f"0.8 x {capacity:.3g} liftings/s (the batched record) / "
                     f"{mean_budget:.3g} liftings (mean budget)")
    reqs = serve.make_requests(a.requests, seed=a.seed, rate=rate,
                               budget_range=tuple(a.serve_budget))
    t0 = time.perf_counter()
    serve.prepare(reqs)
    t_prep = time.perf_counter() - t0
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(hbm_budget_bytes=int(free * 0.6), stream=stream, release_starts=True)
    try:
        with ClockSampler(clk_index) as clk:
            st = srv.serve(reqs)
    finally:
        srv.close()
    summ = st.summary()
    # one at a time: a sample stratified over N (sorted by N, evenly spaced)
    order = sorted(reqs, key=lambda r: r.n)
    picks = [order[int(q)] for q in np.linspace(0, len(order) - 1, 8).round()]
    serve.prepare(picks)
    one_lifts, one_ms = 0, 0.0
    for r in picks:
        got, ms = serve.run_alone_timed(r, undo_cap=srv.undo_cap, stream=stream)
        one_lifts += got
        one_ms += ms
    one = one_lifts / (one_ms / 1e3)
    return {
        "metric": "served liftings/s (device) with p50/p99 request latency",
        "value": summ["liftings_per_s_device"], "unit": "liftings/s",
        "config": {"workload": f"{a.requests} requests (the recipe: 10^4), Poisson "
                               f"{rate:.3g}/s, N log-uniform [4096, 4194304] (lattice), eta "
                               f"U[0.62, 0.72], k = sqrt(N), budget log-uniform "
                               f"[{a.serve_budget[0]:g}, {a.serve_budget[1]:g}] liftings; "
                               f"fewer requests than the recipe to stay within minutes",
                   "rate_per_s": rate, "rate_from": rate_from, "seed": a.seed},
        "serve": summ, "prepare_s": t_prep,
        "one_at_a_time": {"value": one, "unit": "liftings/s",
                          "sample_requests": len(picks),
                          "sample": "8 requests stratified over N (sorted by N, evenly "
                                    "spaced), each alone to its budget",
                          "liftings": one_lifts, "device_ms": one_ms},
        "served_over_one_at_a_time": summ["liftings_per_s_device"] / one if one else None,
        "clocks": clk.summary()}


def run_batched_bench(a):
    import torch

    from paper_2004_11040_gb300 import build
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    r = batched_record(a, torch.cuda.current_stream(), local)
    if rank != 0:
        return
    r.update({"metric": "batched liftings/s over all replicas", "n_gpus": ws,
              "steps": r["launches"], "warmup": 0,
              "ms_per_step": r["device_ms"] / max(1, r["launches"]), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
              "gpu_launches": r["launches"]})
    print(json.dumps(r), flush=True)


def run_serve_bench(a):
    import torch

    from paper_2004_11040_gb300 import build
    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    r = served_record(a, torch.cuda.current_stream(), local)
    if rank != 0:
        return
    r.update({"n_gpus": ws, "steps": r["serve"]["slices"], "warmup": 0,
              "ms_per_step": r["serve"]["device_ms"] / max(1, r["serve"]["slices"]),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f64", "data": "synthetic", "gpu_launches": r["serve"]["slices"]})
    print(json.dumps(r), flush=True)


def run_conflicts(a):
    """Sec. 3.4's birthday scaling: per claim window, the fraction of chains
    that met another chain (their parallel pass stopped at another chain's
    strong claim) and the fraction of windows that needed a repair, against
    k^2 / N, for N = 128^2 (k = 128) and N = 1024^2 (k = 256 .. 16384), at
    W = 1, 16 and 64 claim windows per leg (the finer the windows, the fewer
    chains meet inside one), cell scan and constraint graph."""
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
    modes = [("cells", 1), ("cells", 16), ("cells", 64), ("graph", 1), ("graph", 16)]
    if a.search == "graph":
        modes = [q for q in modes if q[0] == "graph"]
    out = []
    for m, eta, k in points:
        start = synth.lattice_start(m, eta, k, seed=a.seed)
        for search, windows in modes:
            graph = search == "graph"
            sysm = ecmc.System(start.x, start.y, start.active, start.box, a.ell, stream=stream,
                               windows=windows, graph=graph,
                               cells_per_side=m if a.cells == "lattice" else 0)
            t0 = time.perf_counter()
            while sysm.stats()["liftings"] < a.target:
                sysm.run(50)
            st = sysm.stats()
            sysm.close()
            legs = st["legs"]
            nw = legs * windows
            out.append({"N": m * m, "eta": eta, "k": k, "n_over_sqrtN": k / m,
                        "k2_over_N": k * k / (m * m), "search": search,
                        "claim_windows": windows, "legs": legs, "liftings": st["liftings"],
                        "met_chains_per_window_per_chain": st["blocked_chains"] / nw / k,
                        "conflict_windows_per_window": st["conflict_windows"] / nw,
                        "conflict_legs_per_leg": st["conflict_legs"] / legs,
                        "repaired_chains_per_leg_per_chain": st["repaired_chains"] / legs / k,
                        "liftings_per_s": st["liftings"] / (st["device_ms"] / 1e3),
                        "horizon_asserts": st["horizon_asserts"],
                        "order_errors": st["order_errors"],
                        "wall_s": time.perf_counter() - t0})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "chains meeting per claim window vs k^2/N", "unit": "fraction",
                      "n_gpus": 1, "data": "synthetic", "dtype": "f64",
                      "config": {"workload": "jittered square lattices, ell = 1, v = +x",
                                 "cells": a.cells,
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
