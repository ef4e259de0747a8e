"""The serving loop's host logic on the CPU (paper_2004_11040_gb300/serve.py),
with the library replaced by a fake: admission in arrival order while the
device-memory budget allows, one oversized request alone, retirement at the
first breakpoint where a request's budget is met, the latency books, and the
request stream's recipe. The device side of the same loop (results equal to a
request run alone) is tests/test_gpu_serving.py."""
import math
import time

import numpy as np
import pytest

from paper_2004_11040_gb300 import serve

PER_LEG = 3  # liftings per chain and leg in the fake


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeLib:
    """ecmc.System and the batch calls: every system makes PER_LEG * k
    liftings a leg and stops at the first leg end where its budget is met;
    a slice takes 1 ms per leg of its longest system."""

    def __init__(self, clock):
        self.clock = clock
        self.systems = {}
        self.next_id = 1
        self.slices = []
        lib = self

        class System:
            def __init__(self, x, y, active, box, ell, **kw):
                self.ctx = lib.next_id
                lib.next_id += 1
                self.k = len(active)
                self.n = len(x)
                self.closed = False
                lib.systems[self.ctx] = self

            def positions(self):
                return ("positions", self.ctx)

            def close(self):
                assert not self.closed
                self.closed = True

        self.System = System

    def batch_create(self, stream=None):
        return "batch"

    def batch_destroy(self, b):
        pass

    def batch_run(self, batch, ctxs, max_legs, budgets=None):
        lifts = np.zeros(len(ctxs), dtype=np.int64)
        legs = np.zeros(len(ctxs), dtype=np.int32)
        for q, c in enumerate(ctxs):
            s = self.systems[c]
            assert not s.closed
            per = PER_LEG * s.k
            for _ in range(max_legs):
                lifts[q] += per
                legs[q] += 1
                if budgets is not None and budgets[q] > 0 and lifts[q] >= budgets[q]:
                    break
        self.slices.append(len(ctxs))
        ms = float(legs.max()) if len(legs) else 0.0
        self.clock.t += ms / 1e3
        return lifts, legs, ms


@pytest.fixture
def fake(monkeypatch):
    clock = FakeClock()
    lib = FakeLib(clock)
    monkeypatch.setattr(serve.ecmc, "System", lib.System)
    monkeypatch.setattr(serve.ecmc, "ecmc_batch_create", lib.batch_create)
    monkeypatch.setattr(serve.ecmc, "ecmc_batch_destroy", lib.batch_destroy)
    monkeypatch.setattr(serve.ecmc, "ecmc_batch_run", lib.batch_run)
    # device bytes of a request: 100 per disk (the library's own count is
    # checked against cudaMemGetInfo on the GPU)
    monkeypatch.setattr(serve, "device_bytes", lambda n, k, box, **kw: 100 * int(n))

    def sleep(dt):
        clock.t += max(dt, 1e-4)

    monkeypatch.setattr(time, "sleep", sleep)
    return clock, lib


def _stream(count=120, seed=3, rate=200.0):
    reqs = serve.make_requests(count, seed, rate, n_range=(1024, 4096),
                               budget_range=(1e3, 2e5))
    serve.prepare(reqs)
    return reqs


def test_every_request_completes_at_its_first_breakpoint(fake):
    clock, lib = fake
    reqs = _stream()
    srv = serve.Server(hbm_budget_bytes=20 * 100 * 4096, slice_legs=4, keep_results=True)
    st = srv.serve(reqs, clock=clock)
    srv.close()
    assert st.completed == len(reqs)
    assert all(s.closed for s in lib.systems.values())
    assert len(lib.systems) == len(reqs)  # one context per request
    for r in reqs:
        per = PER_LEG * r.k
        assert r.budget <= r.liftings < r.budget + per, (r.rid, r.budget, r.liftings)
        assert r.liftings == r.legs * per
        assert r.arrival <= r.admitted <= r.done
        assert r.result is not None and r.result[0] == "positions"
    assert st.liftings == sum(r.liftings for r in reqs)
    assert st.slices == len(lib.slices)


def test_admission_in_arrival_order_within_the_budget(fake):
    clock, lib = fake
    reqs = _stream(count=150, rate=1e4)  # a burst: requests queue
    budget = 6 * 100 * 4096
    srv = serve.Server(hbm_budget_bytes=budget, slice_legs=2)
    st = srv.serve(reqs, clock=clock)
    srv.close()
    assert st.peak_bytes <= budget
    assert st.peak_resident >= 2  # several systems share the slices
    order = sorted(reqs, key=lambda r: (r.admitted, r.arrival))
    assert [r.rid for r in order] == [r.rid for r in sorted(reqs)]  # first come, first admitted
    # the books: latencies and queue waits of every request
    lat = sorted(r.done - r.arrival for r in reqs)
    assert sorted(st.latencies) == pytest.approx(lat)
    assert all(w >= 0 for w in st.queue_waits)
    summ = st.summary()
    assert summ["p50_latency_s"] == pytest.approx(float(np.percentile(lat, 50)))
    assert summ["p99_latency_s"] == pytest.approx(float(np.percentile(lat, 99)))
    assert summ["completed"] == len(reqs)


def test_max_resident_bounds_the_batch(fake):
    clock, lib = fake
    reqs = _stream(count=60, rate=1e4)
    srv = serve.Server(hbm_budget_bytes=1 << 40, slice_legs=1, max_resident=5)
    st = srv.serve(reqs, clock=clock)
    srv.close()
    assert st.completed == len(reqs)
    assert max(lib.slices) <= 5 and st.peak_resident == 5


def test_an_oversized_request_runs_alone(fake):
    clock, lib = fake
    reqs = _stream(count=20, rate=1e4)
    big = max(reqs, key=lambda r: r.n)
    budget = 100 * big.n - 1  # the largest request alone is over the budget
    srv = serve.Server(hbm_budget_bytes=budget, slice_legs=3)
    st = srv.serve(reqs, clock=clock)
    srv.close()
    assert st.completed == len(reqs)
    # the oversized one was admitted only with nothing else resident
    for r in reqs:
        if r is big:
            others = [q for q in reqs if q is not big and q.admitted <= r.admitted < q.done]
            assert not others
    assert st.peak_bytes <= max(budget, 100 * big.n)


def test_request_stream_recipe():
    a = serve.make_requests(400, 7, rate=20.0)
    b = serve.make_requests(400, 7, rate=20.0)
    assert [(r.arrival, r.n, r.eta, r.budget, r.k) for r in a] == \
           [(r.arrival, r.n, r.eta, r.budget, r.k) for r in b]  # seeded
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    # Poisson arrivals: exponential gaps of mean 1 / rate (400 gaps: within 20 %)
    assert abs(np.mean(np.diff(arr)) - 1.0 / 20.0) < 0.2 / 20.0
    for r in a:
        m = int(round(math.sqrt(r.n)))
        assert m * m == r.n and r.k == m
        assert 4096 <= r.n <= 4_194_304  # M = round(sqrt(N)) stays within the range
        assert 0.62 <= r.eta <= 0.72
        assert 1e5 <= r.budget <= 1e8


def test_mean_budget_is_the_log_uniform_mean():
    a, b = 1e5, 1e8
    # the mean of exp(U(ln a, ln b)) by quadrature
    u = np.linspace(math.log(a), math.log(b), 200001)
    q = np.trapezoid(np.exp(u), u) / (math.log(b) - math.log(a))
    assert serve.Server.mean_budget((a, b)) == pytest.approx(q, rel=1e-6)
    assert serve.Server.mean_budget((5.0, 5.0)) == 5.0
