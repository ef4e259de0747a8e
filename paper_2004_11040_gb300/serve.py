"""Continuous-batching service for independent ECMC runs on one GPU.

Each request is a whole ECMC job: a hard-disk system (N, eta, seed) and a
budget of liftings. Requests arrive over time; the server keeps every admitted
system resident on the device and advances all of them together with one
persistent launch per slice (ecmc_batch_run). Between slices it retires the
systems that reached their budget (stopping, like ecmc_run_to_breakpoint, at
the first breakpoint where the budget is met) and admits new arrivals while
their device memory fits the HBM budget. A system's result does not depend on
which others shared its slices: systems share no state, so a request gives the
same configuration alone and in the mix.
"""
from __future__ import annotations

import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import ecmc, synth

def device_bytes(n: int, k: int, box: float, d: float = 1.0, undo_cap: int = 1024,
                 log_cap: int = 0, cells_per_side: int = 0, ell: float = 1.0,
                 graph: bool = False) -> int:
    """Device memory an ECMC context of these parameters holds, as the
    library computes it without allocating (ecmc_context_bytes): the same
    number its ecmc_stats reports as device_bytes once created."""
    flags = (ecmc.ECMC_LOG_LIFTINGS if log_cap else 0) | (ecmc.ECMC_GRAPH if graph else 0)
    p = ecmc.ecmc_params(int(n), float(box), float(d), float(ell), int(k), int(cells_per_side),
                         flags, int(undo_cap), int(log_cap), 1, 0)
    return ecmc.ecmc_context_bytes(p)


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    n: int = field(compare=False)
    eta: float = field(compare=False)
    seed: int = field(compare=False)
    budget: int = field(compare=False)
    k: int = field(compare=False, default=0)
    start: synth.Start | None = field(compare=False, default=None, repr=False)
    admitted: float = field(compare=False, default=math.nan)
    done: float = field(compare=False, default=math.nan)
    liftings: int = field(compare=False, default=0)
    legs: int = field(compare=False, default=0)
    result: tuple | None = field(compare=False, default=None, repr=False)


def make_requests(count: int, seed: int, rate: float, n_range=(4096, 4_194_304),
                  eta_range=(0.62, 0.72), budget_range=(1e5, 1e8)) -> list[Request]:
    """Seeded request stream: Poisson arrivals at `rate` per second, N and the
    budget log-uniform, eta uniform; the lattice side is M = round(sqrt(N)),
    N := M^2, with k = M chains."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for q in range(count):
        t += float(rng.exponential(1.0 / rate)) if rate > 0 else 0.0
        n_t = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        m = synth.lattice_m_for(int(n_t))
        eta = float(rng.uniform(*eta_range))
        budget = int(math.exp(rng.uniform(math.log(budget_range[0]), math.log(budget_range[1]))))
        out.append(Request(arrival=t, rid=q, n=m * m, eta=eta, seed=seed * 100003 + q,
                           budget=budget, k=m))
    return out


def prepare(reqs: list[Request]) -> None:
    """Builds each request's seeded start (client side, before it arrives)."""
    for r in reqs:
        m = int(round(math.sqrt(r.n)))
        r.start = synth.lattice_start(m, r.eta, r.k, seed=r.seed)


@dataclass
class ServeStats:
    wall_s: float
    device_ms: float
    liftings: int
    slices: int
    completed: int
    latencies: list[float]
    queue_waits: list[float]
    peak_resident: int
    peak_bytes: int

    def summary(self) -> dict:
        lat = np.asarray(self.latencies)
        wait = np.asarray(self.queue_waits)
        return {
            "completed": self.completed,
            "liftings": self.liftings,
            "wall_s": self.wall_s,
            "device_ms": self.device_ms,
            "slices": self.slices,
            "liftings_per_s_wall": self.liftings / self.wall_s if self.wall_s else 0.0,
            "liftings_per_s_device": self.liftings / (self.device_ms / 1e3) if self.device_ms else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "p50_queue_s": float(np.percentile(wait, 50)) if wait.size else None,
            "peak_resident_requests": self.peak_resident,
            "peak_device_bytes": self.peak_bytes,
        }


class Server:
    """Admits requests by device-memory budget and runs slices of legs."""

    def __init__(self, hbm_budget_bytes: int, ell: float = 1.0, slice_legs: int = 8,
                 max_resident: int = 4096, undo_cap: int = 1024, stream=None,
                 keep_results: bool = False, cells: str = "lattice",
                 release_starts: bool = False, graph: bool = False):
        self.hbm_budget = int(hbm_budget_bytes)
        self.cells = cells
        self.ell = ell
        self.slice_legs = slice_legs
        self.max_resident = max_resident
        self.undo_cap = undo_cap
        self.stream = stream
        self.keep_results = keep_results
        # drop a request's host copy of its start once it is on the device
        self.release_starts = release_starts
        # constraint-graph contexts (a batch holds one kind only)
        self.graph = graph
        self.batch = ecmc.ecmc_batch_create(stream)

    def close(self):
        if self.batch:
            ecmc.ecmc_batch_destroy(self.batch)
            self.batch = None

    def _cells(self, r: Request) -> int:
        # "lattice": one cell per site of the start lattice (every row of disks
        # inside one cell row, where the row pass applies); else the default
        return int(r.start.m) if self.cells == "lattice" else 0

    def need(self, r: Request) -> int:
        """Device bytes request r will hold (from the library, no allocation)."""
        return device_bytes(r.n, r.k, r.start.box, undo_cap=self.undo_cap,
                            cells_per_side=self._cells(r), ell=self.ell, graph=self.graph)

    @staticmethod
    def mean_budget(budget_range) -> float:
        """Mean of a log-uniform budget on [a, b]: (b - a) / ln(b / a)."""
        a, b = float(budget_range[0]), float(budget_range[1])
        return a if b <= a else (b - a) / math.log(b / a)

    def _admit(self, r: Request):
        s = r.start
        return ecmc.System(s.x, s.y, s.active, s.box, self.ell, undo_cap=self.undo_cap,
                           stream=self.stream, cells_per_side=self._cells(r), graph=self.graph)

    def serve(self, reqs: list[Request], clock=time.perf_counter) -> ServeStats:
        """Runs the stream to completion; arrival times are seconds after start."""
        arrivals = sorted(reqs)
        pending: list[Request] = []  # arrived, waiting for memory (FIFO)
        running: dict[int, tuple[Request, ecmc.System, int]] = {}
        used = 0
        t0 = clock()
        nxt = 0
        dev_ms = 0.0
        lifts_total = 0
        slices = 0
        peak_res = 0
        peak_bytes = 0
        lat, waits = [], []
        while nxt < len(arrivals) or pending or running:
            now = clock() - t0
            while nxt < len(arrivals) and arrivals[nxt].arrival <= now:
                pending.append(arrivals[nxt])
                nxt += 1
            # admission: FIFO while the device budget and the slot count allow
            while pending and len(running) < self.max_resident:
                r = pending[0]
                need = self.need(r)
                if running and used + need > self.hbm_budget:
                    break
                pending.pop(0)
                sysm = self._admit(r)
                if self.release_starts:
                    r.start = None
                r.admitted = clock() - t0
                running[r.rid] = (r, sysm, need)
                used += need
            peak_res = max(peak_res, len(running))
            peak_bytes = max(peak_bytes, used)
            if not running:
                if nxt < len(arrivals):
                    time.sleep(max(0.0, min(0.01, arrivals[nxt].arrival - (clock() - t0))))
                continue
            items = list(running.values())
            budgets = [r.budget - r.liftings for r, _, _ in items]
            lifts, legs, ms = ecmc.ecmc_batch_run(self.batch, [s.ctx for _, s, _ in items],
                                                  self.slice_legs, budgets)
            slices += 1
            dev_ms += ms
            now = clock() - t0
            for (r, sysm, need), nl, ng in zip(items, lifts, legs):
                r.liftings += int(nl)
                r.legs += int(ng)
                lifts_total += int(nl)
                if r.liftings >= r.budget:
                    if self.keep_results:
                        r.result = sysm.positions()
                    sysm.close()
                    r.done = clock() - t0
                    lat.append(r.done - r.arrival)
                    waits.append(r.admitted - r.arrival)
                    del running[r.rid]
                    used -= need
        wall = clock() - t0
        return ServeStats(wall_s=wall, device_ms=dev_ms, liftings=lifts_total, slices=slices,
                          completed=len(lat), latencies=lat, queue_waits=waits,
                          peak_resident=peak_res, peak_bytes=peak_bytes)


def run_alone(r: Request, ell: float = 1.0, undo_cap: int = 1024, stream=None,
              cells: str = "lattice", graph: bool = False):
    """The same request on its own: ecmc_run_to_breakpoint with the budget."""
    s = r.start
    sysm = ecmc.System(s.x, s.y, s.active, s.box, ell, undo_cap=undo_cap, stream=stream,
                       cells_per_side=int(s.m) if cells == "lattice" else 0, graph=graph)
    total = 0
    while total < r.budget:
        before = sysm.stats()["liftings"]
        sysm.run(1 << 20, event_budget=r.budget - total)
        total += sysm.stats()["liftings"] - before
    out = sysm.positions()
    sysm.close()
    return out, total


def run_alone_timed(r: Request, ell: float = 1.0, undo_cap: int = 1024, stream=None,
                    cells: str = "lattice") -> tuple[int, float]:
    """The same request on its own, as few launches as the budget allows
    (ecmc_run_to_breakpoint with the budget); returns (liftings, device ms)."""
    s = r.start
    sysm = ecmc.System(s.x, s.y, s.active, s.box, ell, undo_cap=undo_cap, stream=stream,
                       cells_per_side=int(s.m) if cells == "lattice" else 0)
    try:
        while sysm.stats()["liftings"] < r.budget:
            sysm.run(1 << 20, event_budget=r.budget - sysm.stats()["liftings"])
        st = sysm.stats()
    finally:
        sysm.close()
    return st["liftings"], st["device_ms"]
