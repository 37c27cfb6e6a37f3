"""The autotuners' host logic on the CPU: with a fake batch, context and
query whose calls advance a fake stream clock by a cost per candidate, and
CUDA events that read that clock, each tuner keeps the cheapest candidate,
sets it, writes it to the JSON cache under the shape's signature, and a
second call takes it from the cache without timing.  Unreadable caches are
ignored; the cache file is replaced whole."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

from paper_2206_10435_gb300 import autotune as A
from paper_2206_10435_gb300 import gj


class FakeStream:
    def __init__(self):
        self.t = 0.0

    def synchronize(self):
        pass


class FakeEvent:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream):
        self.t = stream.t

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


@pytest.fixture()
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)


class FakeCtx:
    def __init__(self):
        self.device = 0
        self.stream = FakeStream()
        self.options = {}
        self.calls = []

    def set_option(self, opt, value):
        self.options[opt] = value
        self.calls.append((opt, value))


class FakeBatch:
    def __init__(self, cost):
        self.ctx = FakeCtx()
        self.cost = cost
        self.n_rows, self.n_relations, self.levels, self.key_bits = 3_000_000, 40, 5, 41
        self.grid_mult = None
        self.runs = 0

    def set_grid_mult(self, m):
        self.grid_mult = m

    def run(self, use_graph=True):
        self.runs += 1
        self.ctx.stream.t += self.cost[self.grid_mult]


class FakeQuery:
    def __init__(self, ctx, opt, cost, total=123_456):
        self.ctx, self.opt, self.cost, self.total = ctx, opt, cost, total
        self.n_groups = [1000, 4000, 50]
        self.n_rel = 3
        self.parent = [-1, 0, 1]
        self.col_width = [4, 4, 4, 4, 8]
        self.calls = 0

    def _tick(self):
        self.calls += 1
        self.ctx.stream.t += self.cost[self.ctx.options[self.opt]]

    def alloc_columns(self, n):
        return [None] * len(self.col_width)

    def desummarize(self, row0, n, out=None):
        self._tick()
        return out

    def summarize(self):
        self._tick()
        return self.total


def test_batch_tuner_keeps_the_cheapest_grid_and_caches_it(fake_cuda, tmp_path):
    cache = str(tmp_path / "t.json")
    b = FakeBatch({1: 9.0, 2: 5.0, 4: 2.0, 8: 3.0, 16: 7.0})
    r = A.tune_batch(b, reps=2, cache_path=cache)
    assert r["grid_mult"] == 4 and b.grid_mult == 4 and not r["cached"]
    assert r["ms"] == pytest.approx(2.0)
    assert r["candidates_ms"] == {"1": 9.0, "2": 5.0, "4": 2.0, "8": 3.0, "16": 7.0}
    stored = json.load(open(cache))
    assert list(stored) == [A.signature(b, "FakeGPU")]
    assert A.signature(b, "FakeGPU") == "FakeGPU|rows2^22|rel40|lv5|bits41"
    b2 = FakeBatch({m: 1.0 for m in A.CANDIDATES})
    r2 = A.tune_batch(b2, cache_path=cache)
    assert r2["cached"] and r2["grid_mult"] == 4 and b2.grid_mult == 4 and b2.runs == 0
    # use_cache=False times again and leaves the file alone
    r3 = A.tune_batch(b2, reps=1, cache_path=cache, use_cache=False)
    assert not r3["cached"] and b2.runs > 0
    assert json.load(open(cache)) == stored


def test_emit_tuner_keeps_the_cheapest_rows_per_thread(fake_cuda, tmp_path):
    cache = str(tmp_path / "t.json")
    ctx = FakeCtx()
    q = FakeQuery(ctx, gj.GJ_OPT_EMIT_ROWS_PER_THREAD, {2: 4.0, 4: 3.0, 8: 1.5})
    r = A.tune_emit(ctx, q, window=1 << 20, reps=3, cache_path=cache)
    assert r["rpt"] == 8 and ctx.options[gj.GJ_OPT_EMIT_ROWS_PER_THREAD] == 8
    assert set(r["candidates_ms"]) == {"2", "4", "8"}
    key = A.emit_signature(q, "FakeGPU", min(1 << 20, q.total))
    assert key in json.load(open(cache))
    ctx2 = FakeCtx()
    q2 = FakeQuery(ctx2, gj.GJ_OPT_EMIT_ROWS_PER_THREAD, {2: 0.0, 4: 0.0, 8: 9.0})
    r2 = A.tune_emit(ctx2, q2, window=1 << 20, cache_path=cache)
    assert r2["cached"] and r2["rpt"] == 8 and q2.calls == 0
    # an empty result is not timed
    q3 = FakeQuery(FakeCtx(), gj.GJ_OPT_EMIT_ROWS_PER_THREAD, {}, total=0)
    assert "skipped" in A.tune_emit(q3.ctx, q3, cache_path=cache)


@pytest.mark.parametrize("triangle", [False, True])
def test_summary_tuner_keeps_the_cheapest_option(fake_cuda, tmp_path, triangle):
    cache = str(tmp_path / "t.json")
    opt = gj.GJ_OPT_TRIANGLE_INTERSECT if triangle else gj.GJ_OPT_DOWN_COMBINE
    name = "triangle_intersect" if triangle else "down_combine"
    cost = {1: 2.0, 2: 0.5} if triangle else {0: 1.0, 1: 0.25, 2: 3.0}
    ctx = FakeCtx()
    q = FakeQuery(ctx, opt, cost)
    r = A.tune_summary(ctx, q, triangle=triangle, reps=2, cache_path=cache)
    best = min(cost, key=cost.get)
    assert r[name] == best and ctx.options[opt] == best and not r["cached"]
    assert json.load(open(cache))[A.summary_signature(q, "FakeGPU", name)][name] == best
    ctx2 = FakeCtx()
    r2 = A.tune_summary(ctx2, FakeQuery(ctx2, opt, cost), triangle=triangle, cache_path=cache)
    assert r2["cached"] and ctx2.options[opt] == best


def test_summary_tuner_refuses_options_that_disagree(fake_cuda, tmp_path):
    ctx = FakeCtx()
    q = FakeQuery(ctx, gj.GJ_OPT_DOWN_COMBINE, {0: 1.0, 1: 1.0, 2: 1.0})
    totals = iter([5, 5, 5, 6, 6, 6, 5, 5, 5])
    q.summarize = lambda: (q._tick(), next(totals))[1]
    with pytest.raises(RuntimeError):
        A.tune_summary(ctx, q, reps=2, cache_path=str(tmp_path / "t.json"))


def test_signatures_separate_shapes():
    ctx = FakeCtx()
    a = FakeQuery(ctx, 0, {})
    b = FakeQuery(ctx, 0, {})
    b.parent = [-1, 0, 0]
    assert A.summary_signature(a, "G", "down_combine") != A.summary_signature(b, "G", "down_combine")
    assert A.summary_signature(a, "G", "down_combine") != A.summary_signature(a, "H", "down_combine")
    assert A.emit_signature(a, "G", 1 << 20) != A.emit_signature(a, "G", 1 << 24)


def test_cache_files(tmp_path):
    p = str(tmp_path / "sub" / "c.json")
    assert A._load_cache(p, True) == {}
    A._store_cache(p, {"k": {"v": 1}})
    assert A._load_cache(p, True) == {"k": {"v": 1}}
    assert A._load_cache(p, False) == {}
    assert os.listdir(os.path.dirname(p)) == ["c.json"]    # no temporary left behind
    for bad in ("{not json", "[1, 2]"):
        with open(p, "w") as f:
            f.write(bad)
        assert A._load_cache(p, True) == {}
