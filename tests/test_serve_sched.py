"""Scheduler of the serving loop, with a fake engine (no GPU): admission
under the memory budget, FIFO order, slot concurrency, rejection; the
latency statistics of the native server's results and the Poisson arrival
process of the serving benchmark."""
import threading
import time

from paper_2206_10435_gb300.serve import Engine, Request, Server, latency_stats, poisson_arrivals, run_stream


class FakeEngine(Engine):
    def __init__(self, sizes, dur=0.01):
        self.sizes = sizes
        self.dur = dur
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.order = []

    def plan(self, req):
        return None, self.sizes[req.query]

    def run(self, req, slot):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.order.append(req.rid)
        time.sleep(self.dur)
        req.total = req.query
        req.t_summary = time.perf_counter()
        req.t_chunk = time.perf_counter()
        with self.lock:
            self.running -= 1


def test_budget_is_never_exceeded_and_order_is_fifo():
    sizes = {i: (i % 5 + 1) * 10 for i in range(40)}
    eng = FakeEngine(sizes, dur=0.005)
    srv = Server(eng, n_slots=8, hbm_budget=100)
    reqs = [Request(i, i) for i in range(40)]
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert all(r.status == "ok" for r in reqs)
    assert srv.peak_used <= 100
    assert srv.used == 0 and srv.in_flight == 0
    assert sorted(eng.order) == list(range(40))
    assert eng.order[:3] == [0, 1, 2]          # admitted in arrival order
    assert eng.max_running > 1                 # requests overlap


def test_slots_bound_concurrency():
    eng = FakeEngine({i: 1 for i in range(30)}, dur=0.01)
    srv = Server(eng, n_slots=3, hbm_budget=10**9)
    for i in range(30):
        srv.submit(Request(i, i))
    srv.drain()
    assert eng.max_running <= 3 and srv.peak_in_flight <= 3


def test_oversized_request_is_rejected_others_served():
    eng = FakeEngine({0: 5, 1: 500, 2: 5}, dur=0.001)
    srv = Server(eng, n_slots=2, hbm_budget=100)
    reqs = [Request(i, i) for i in range(3)]
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert [r.status for r in reqs] == ["ok", "rejected", "ok"]


def test_poisson_stream_and_stats():
    eng = FakeEngine({i: 1 for i in range(50)}, dur=0.002)
    srv = Server(eng, n_slots=4, hbm_budget=10**9)
    offs = poisson_arrivals(2000.0, 50, seed=1)
    reqs = run_stream(srv, list(range(50)), offs)
    st = latency_stats(reqs)
    assert st["completed"] == 50 and st["p99_first_chunk_ms"] >= st["p50_first_chunk_ms"] > 0


def test_native_stats_of_known_times():
    from paper_2206_10435_gb300.serve import native_latency_stats
    # request i arrives at i ms; summary +1 ms, first chunk +2 ms, last chunk
    # +(3 + i % 4) ms; every 10th request failed (status 3, out of memory),
    # request 5 overflowed (status 4, still answered)
    res = []
    for i in range(100):
        t = i / 1000.0
        res.append({"status": 3 if i % 10 == 9 else (4 if i == 5 else 0), "t_arrival": t,
                    "t_summary": t + 0.001, "t_chunk": t + 0.002, "t_last": t + (3 + i % 4) / 1000.0,
                    "rows": 10})
    st = native_latency_stats(res)
    assert st["completed"] == 90 and st["failed"] == 10 and st["rows_streamed"] == 900
    assert abs(st["p50_summary_ms"] - 1.0) < 1e-9 and abs(st["p99_first_chunk_ms"] - 2.0) < 1e-9
    assert 3.0 <= st["p50_last_chunk_ms"] <= 6.0 and abs(st["p99_last_chunk_ms"] - 6.0) < 1e-9
    # the span runs from the first arrival (0 ms) to the last finished chunk
    # of a completed request (request 98: 98 + 5 ms)
    assert abs(st["qps"] - 90 / 0.103) < 1e-6 and abs(st["rows_per_s"] - 900 / 0.103) < 1e-6
    assert native_latency_stats([dict(res[9])]) == {"completed": 0}


def test_poisson_arrivals_have_the_offered_rate():
    offs = poisson_arrivals(1000.0, 20_000, seed=3)
    gaps = offs[1:] - offs[:-1]
    assert (gaps > 0).all()
    assert abs(offs[-1] / 20_000 - 1e-3) < 3e-5            # mean gap within 3%
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05      # exponential: sd = mean
