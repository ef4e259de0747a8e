"""Batched replicas and the continuous-batching server: a system's result
does not depend on which others share its launches. Every replica or request
must end, bit for bit, where the same system run alone ends (and, for small
ones, where the oracle ends)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_11040_gb300 import batch, ecmc, serve

pytestmark = pytest.mark.gpu


def _final(sysm):
    x, y, t, a = sysm.positions()
    return x, t, a


def test_batched_replicas_equal_alone_and_oracle():
    reps = batch.make_replicas(12, seed=5, n_range=(256, 4096))
    budget = 6000
    systems = batch.create(reps)
    lifts, ms, launches = batch.run_batched(systems, budget, legs_per_launch=3)
    assert ms > 0 and launches >= 1
    finals = [_final(s) for s in systems]
    per_rep = [s.stats()["liftings"] for s in systems]
    for s in systems:
        s.close()
    assert lifts == sum(per_rep)
    plain = batch.create(reps)
    p_lifts, _, _ = batch.run_plain(plain, budget, legs_per_launch=3)
    assert p_lifts == lifts
    for q, (s, f) in enumerate(zip(plain, finals)):
        g = _final(s)
        assert all(np.array_equal(u, v) for u, v in zip(f, g)), q
        s.close()
    # the two smallest against the oracle: the stopping leg and the state
    for q in np.argsort([r.start.n for r in reps])[:2]:
        r = reps[q]
        _, legs = O.run_legs(r.start.x, r.start.y, r.start.active, r.start.box, r.ell, 64)
        cum = np.cumsum([g.lifts for g in legs])
        stop = int(np.searchsorted(cum, budget) + 1)
        last, _ = O.run_legs(r.start.x, r.start.y, r.start.active, r.start.box, r.ell, stop)
        assert per_rep[q] == cum[stop - 1]
        assert np.array_equal(finals[q][0], last.x) and np.array_equal(finals[q][1], last.t)
        assert np.array_equal(finals[q][2], last.active)


def test_autotune_picks_and_caches(tmp_path, monkeypatch):
    reps = batch.make_replicas(8, seed=9, n_range=(1024, 4096))
    cache = str(tmp_path / "tune.json")
    got = batch.autotune(reps, trial_budget=2000, cells_options=("lattice", "default"),
                         search_options=("row", "general", "graph"), legs_options=(2, 8),
                         cache=cache)
    assert got["cells"] in ("lattice", "default") and got["legs_per_launch"] in (2, 8)
    assert got["search"] in ("row", "general", "graph")
    # cells x {row, general} and the graph once, each with both leg counts
    assert len(got["trials"]) == 10 and all(t["liftings_per_s"] > 0 for t in got["trials"])
    assert sum(t["search"] == "graph" for t in got["trials"]) == 2
    # the row pass runs where the cells are aligned with the lattice
    assert any(t["row_windows"] > 0 for t in got["trials"]
               if t["search"] == "row" and t["cells"] == "lattice")
    assert all(t["row_windows"] == 0 for t in got["trials"] if t["search"] != "row")
    again = batch.autotune(reps, cache=cache)  # served from the cache, no trials run
    assert (again["cells"], again["search"], again["legs_per_launch"]) == \
        (got["cells"], got["search"], got["legs_per_launch"])
    # another GPU or library build: the cached choice does not apply
    monkeypatch.setattr(batch, "_hardware_key", lambda: "other-gpu_other-build")
    fresh = batch.autotune(reps, trial_budget=2000, cells_options=("lattice",),
                           search_options=("row",), legs_options=(2,), cache=cache)
    assert len(fresh["trials"]) == 1 and fresh["key"].startswith("other-gpu_other-build")


def test_server_mix_equals_alone():
    reqs = serve.make_requests(10, seed=3, rate=0.0, n_range=(1024, 16384),
                               budget_range=(2e3, 5e4))
    serve.prepare(reqs)
    # a budget that holds about three of them at once forces queueing
    probe = serve.Server(hbm_budget_bytes=1, slice_legs=4)
    need = sorted(probe.need(r) for r in reqs)
    probe.close()
    srv = serve.Server(hbm_budget_bytes=sum(need[-3:]), slice_legs=4, keep_results=True)
    try:
        st = srv.serve(reqs)
    finally:
        srv.close()
    summ = st.summary()
    assert st.completed == len(reqs)
    assert summ["p50_latency_s"] is not None and summ["p99_latency_s"] >= summ["p50_latency_s"]
    assert st.peak_bytes <= sum(need[-3:])
    assert st.liftings == sum(r.liftings for r in reqs)
    for r in reqs:
        assert r.liftings >= r.budget
        (x, y, t, a), total = serve.run_alone(r)
        rx, ry, rt, ra = r.result
        assert total == r.liftings, r.rid
        assert np.array_equal(x, rx) and np.array_equal(t, rt) and np.array_equal(a, ra), r.rid


def test_server_graph_mode_mix_equals_alone():
    """The server with constraint-graph contexts (batched by their own
    kernel): each request ends where the same request alone ends."""
    reqs = serve.make_requests(8, seed=6, rate=0.0, n_range=(1024, 16384),
                               budget_range=(2e3, 5e4))
    serve.prepare(reqs)
    probe = serve.Server(hbm_budget_bytes=1, slice_legs=4, graph=True)
    need = sorted(probe.need(r) for r in reqs)
    probe.close()
    srv = serve.Server(hbm_budget_bytes=sum(need[-3:]), slice_legs=4, keep_results=True,
                       graph=True)
    try:
        st = srv.serve(reqs)
    finally:
        srv.close()
    assert st.completed == len(reqs)
    assert st.peak_bytes <= sum(need[-3:])
    for r in reqs:
        (x, y, t, a), total = serve.run_alone(r, graph=True)
        rx, ry, rt, ra = r.result
        assert total == r.liftings, r.rid
        assert np.array_equal(x, rx) and np.array_equal(t, rt) and np.array_equal(a, ra), r.rid


def test_server_poisson_arrivals_complete():
    reqs = serve.make_requests(6, seed=4, rate=200.0, n_range=(1024, 8192),
                               budget_range=(1e3, 2e4))
    serve.prepare(reqs)
    srv = serve.Server(hbm_budget_bytes=1 << 30, slice_legs=2)
    try:
        st = srv.serve(reqs)
    finally:
        srv.close()
    assert st.completed == 6
    assert all(lat >= 0 for lat in st.latencies)
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)


def test_context_bytes_are_what_a_context_holds():
    """ecmc_context_bytes (nothing allocated) equals the device_bytes of the
    created context, and the device's free memory drops by that much (to the
    allocator's granularity) when the library's cache holds nothing."""
    import torch
    from paper_2004_11040_gb300 import synth
    ecmc.ecmc_set_cache_limit(0)  # every block from cudaMalloc, back by cudaFree
    try:
        _context_bytes_cases(torch, synth)
    finally:
        ecmc.ecmc_set_cache_limit(4 << 30)


def _context_bytes_cases(torch, synth):
    for m, k, cells, graph in ((64, 64, 64, False), (256, 512, 0, False), (512, 512, 512, False),
                               (64, 64, 0, True), (512, 512, 512, True)):
        s = synth.lattice_start(m, 0.70, k, seed=1)
        need = serve.device_bytes(m * m, k, s.box, undo_cap=256, cells_per_side=cells,
                                  graph=graph)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        sysm = ecmc.System(s.x, s.y, s.active, s.box, 1.0, undo_cap=256, cells_per_side=cells,
                           graph=graph)
        sysm.positions()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        got = sysm.stats()["device_bytes"]
        sysm.close()
        assert got == need, (m, got, need)
        drop = free0 - free1
        assert need - (4 << 20) <= drop <= need + (8 << 20), (m, drop, need)

