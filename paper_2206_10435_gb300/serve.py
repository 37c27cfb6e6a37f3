"""Serving loop: join queries arriving as a stream, continuously admitted.

Requests name queries over relations that stay loaded on the device with
their factors built (the paper's pre-built potentials, Section 4.1).  Each
request is answered with its join size and summary and the first chunk of
its result rows (a cursor's first page; later pages are further windows of
the same summary).

Scheduling:
  * a dispatcher releases requests at their arrival times;
  * admission plans a request (no device work when its factors exist),
    estimates the device memory its summary and first chunk need, and admits
    it into a free slot only while the admitted total stays under the HBM
    budget (FIFO, so a large request is not starved by small ones);
  * every slot is a host thread with its own CUDA stream; admitted requests
    run concurrently, so requests that arrive while others are on the GPU
    overlap with them on the device as soon as a slot and memory are free.

Latency is measured from arrival to summary and to the first chunk.
The engine (what runs one request) is separate from the scheduler so the
scheduler's logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    query: object                  # engine-specific description (e.g. relation ids)
    arrival: float = 0.0           # time.perf_counter() at arrival
    est_bytes: int = 0
    plan: object = None
    total: int | None = None
    status: str = "pending"
    t_admit: float = 0.0
    t_summary: float = 0.0
    t_chunk: float = 0.0           # first result chunk out
    t_last: float = 0.0            # last result chunk out
    rows: int = 0                  # result rows streamed
    slot: int = -1
    result: object = None          # engine-specific (checksum or host copy)


class Engine:
    """What the server needs from a backend."""

    def plan(self, req: Request):
        """Host-side planning; returns (plan, estimated device bytes)."""
        raise NotImplementedError

    def run(self, req: Request, slot: int):
        """Runs the request on `slot`; sets req.total, req.t_summary, req.t_chunk."""
        raise NotImplementedError

    def release(self, req: Request):
        pass


class Server:
    def __init__(self, engine: Engine, n_slots: int = 16, hbm_budget: int = 150 * 10**9):
        self.engine = engine
        self.n_slots = n_slots
        self.budget = hbm_budget
        self.used = 0
        self.peak_used = 0
        self.in_flight = 0
        self.peak_in_flight = 0
        self.pending = collections.deque()
        self.done = []
        self.cv = threading.Condition()
        self.stopping = False
        self.errors = []
        self.workers = [threading.Thread(target=self._worker, args=(s,), daemon=True)
                        for s in range(n_slots)]
        for w in self.workers:
            w.start()

    # ------------------------------------------------------------ intake
    def submit(self, req: Request):
        if not req.arrival:
            req.arrival = time.perf_counter()
        req.plan, req.est_bytes = self.engine.plan(req)
        if req.est_bytes > self.budget:
            req.status = "rejected"
            self.engine.release(req)
            with self.cv:
                self.done.append(req)
                self.cv.notify_all()
            return
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()

    # ------------------------------------------------------------ slots
    def _admit(self):
        """Called with the lock held: the head request if it fits, else None."""
        if not self.pending:
            return None
        head = self.pending[0]
        if self.used + head.est_bytes > self.budget and self.in_flight > 0:
            return None
        self.pending.popleft()
        self.used += head.est_bytes
        self.in_flight += 1
        self.peak_used = max(self.peak_used, self.used)
        self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
        head.t_admit = time.perf_counter()
        return head

    def _worker(self, slot: int):
        while True:
            with self.cv:
                req = self._admit()
                while req is None:
                    if self.stopping and not self.pending:
                        return
                    self.cv.wait(0.05)
                    req = self._admit()
            req.slot = slot
            try:
                self.engine.run(req, slot)
                req.status = "ok" if req.status == "pending" else req.status
            except Exception as e:   # recorded, the server keeps serving
                req.status = f"error: {e}"
                self.errors.append(req)
            finally:
                self.engine.release(req)
                with self.cv:
                    self.used -= req.est_bytes
                    self.in_flight -= 1
                    self.done.append(req)
                    self.cv.notify_all()

    def drain(self, timeout: float = 600.0):
        """Waits until every submitted request finished, then stops."""
        end = time.perf_counter() + timeout
        with self.cv:
            while (self.pending or self.in_flight) and time.perf_counter() < end:
                self.cv.wait(0.05)
            self.stopping = True
            self.cv.notify_all()
        for w in self.workers:
            w.join(timeout=5)


def poisson_arrivals(rate: float, n: int, seed: int = 0):
    """n arrival offsets (seconds) of a Poisson process of the given rate."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_stream(server: Server, queries, offsets):
    """Submits queries[i] at start + offsets[i]; returns the requests."""
    reqs = [Request(i, q) for i, q in enumerate(queries)]
    t0 = time.perf_counter()
    for r, off in zip(reqs, offsets):
        delay = t0 + off - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        r.arrival = time.perf_counter()
        server.submit(r)
    server.drain()
    return reqs


def native_latency_stats(results):
    """latency_stats for the result dicts of gj.NativeServer.run."""
    import numpy as np
    ok = [r for r in results if r["status"] in (0, 4)]   # GJ_OK, GJ_ERR_OVERFLOW
    if not ok:
        return {"completed": 0}
    s = np.array([r["t_summary"] - r["t_arrival"] for r in ok]) * 1000
    c = np.array([r["t_chunk"] - r["t_arrival"] for r in ok]) * 1000
    last = np.array([r["t_last"] - r["t_arrival"] for r in ok]) * 1000
    span = max(r["t_last"] for r in ok) - min(r["t_arrival"] for r in ok)
    rows = sum(int(r["rows"]) for r in ok)
    return {"completed": len(ok), "failed": len(results) - len(ok),
            "qps": len(ok) / span if span > 0 else None,
            "rows_streamed": rows, "rows_per_s": rows / span if span > 0 else None,
            "p50_summary_ms": float(np.percentile(s, 50)), "p99_summary_ms": float(np.percentile(s, 99)),
            "p50_first_chunk_ms": float(np.percentile(c, 50)), "p99_first_chunk_ms": float(np.percentile(c, 99)),
            "p50_last_chunk_ms": float(np.percentile(last, 50)), "p99_last_chunk_ms": float(np.percentile(last, 99))}


def latency_stats(reqs):
    import numpy as np
    ok = [r for r in reqs if r.status in ("ok", "overflow")]
    if not ok:
        return {"completed": 0}
    s = np.array([r.t_summary - r.arrival for r in ok]) * 1000
    c = np.array([r.t_chunk - r.arrival for r in ok]) * 1000
    last = np.array([max(r.t_last, r.t_chunk) - r.arrival for r in ok]) * 1000
    span = max(max(r.t_last, r.t_chunk) for r in ok) - min(r.arrival for r in ok)
    rows = sum(r.rows for r in ok)
    return {"completed": len(ok), "rejected": sum(r.status == "rejected" for r in reqs),
            "errors": sum(r.status.startswith("error") for r in reqs),
            "qps": len(ok) / span if span > 0 else None,
            "rows_streamed": rows, "rows_per_s": rows / span if span > 0 else None,
            "p50_summary_ms": float(np.percentile(s, 50)), "p99_summary_ms": float(np.percentile(s, 99)),
            "p50_first_chunk_ms": float(np.percentile(c, 50)), "p99_first_chunk_ms": float(np.percentile(c, 99)),
            "p50_last_chunk_ms": float(np.percentile(last, 50)), "p99_last_chunk_ms": float(np.percentile(last, 99))}


class GJEngine(Engine):
    """Runs a request through the C ABI: plan (gj_query_create with resident
    factors), then on the slot's stream summarise and stream the result rows
    (up to max_rows, 0 = all) chunk by chunk through the slot's buffers."""

    def __init__(self, ctx, n_slots: int, chunk_rows: int = 1 << 20, keep_results: bool = False,
                 max_cols: int = 16, max_rows: int = 0):
        import torch
        from . import gj
        self.torch = torch
        self.gj = gj
        self.ctx = ctx
        self.chunk = chunk_rows
        self.max_rows = max_rows
        self.keep = keep_results
        dev = torch.device("cuda", ctx.device)
        self.streams = [torch.cuda.Stream(dev) for _ in range(n_slots)]
        self.bufs = [None] * n_slots
        self.dev = dev

    def plan(self, req: Request):
        q = self.ctx.query(req.query)          # factors are resident: host work only
        groups = sum(q.n_groups)
        k = q.n_rel
        est = 80 * groups + 2 * min(self.chunk, 1 << 31) * (16 + 4 * k) + (1 << 20)
        return q, est

    def run(self, req: Request, slot: int):
        torch = self.torch
        st = self.streams[slot]
        q = req.plan
        with torch.cuda.stream(st):
            q.set_stream(st)
            try:
                req.total = q.summarize()
            except self.gj.GJError as e:
                if e.status != self.gj.GJ_ERR_OVERFLOW:
                    raise
                req.total = self.gj.SAT
                req.status = "overflow"
            req.t_summary = time.perf_counter()
            if req.status == "pending" and req.total > 0:
                want = min(self.max_rows, req.total) if self.max_rows else req.total
                widths = q.col_width
                buf = self.bufs[slot]
                if buf is None or len(buf) != len(widths) or any(
                        b.element_size() != w for b, w in zip(buf, widths)):
                    buf = [torch.empty(self.chunk, dtype=torch.int32 if w == 4 else torch.int64,
                                       device=self.dev) for w in widths]
                    self.bufs[slot] = buf
                kept = []
                for r0 in range(0, want, self.chunk):
                    cols = q.desummarize(r0, min(self.chunk, want - r0), out=buf)
                    if self.keep:
                        kept.append([c.cpu() for c in cols])
                    if r0 == 0:
                        st.synchronize()
                        req.t_chunk = time.perf_counter()
                req.rows = want
                if self.keep:
                    req.result = [torch.cat([k[i] for k in kept]) for i in range(len(widths))]
            st.synchronize()
            req.t_last = time.perf_counter()
            if not req.t_chunk:
                req.t_chunk = req.t_last

    def release(self, req: Request):
        if req.plan is not None:
            req.plan.close()
            req.plan = None
