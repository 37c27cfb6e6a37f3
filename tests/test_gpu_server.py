"""The native serving runtime (gj_server_*): join sizes against the oracle,
and every request's first result chunk (by its hash) identical when the
request runs alone and when it runs mixed with concurrent requests."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pool(n=20, seed=8):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        k = int(rng.integers(2, 6))
        rows = rng.integers(100, 20000, size=k)
        doms = rng.integers(5, 2000, size=k + 1)
        s = float(rng.uniform(0, 1.4))
        qs.append(G.chain_query(f"p{i}", rows, doms, [s] * (k + 1), np.int64 if i % 2 else np.int32,
                                2000 + i))
    return qs


def test_native_server_alone_equals_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    ctx = gj.Context(0, torch.cuda.Stream())
    pool = _pool()
    ref = [O.count(q).total for q in pool]
    ids = [gj.load_query(ctx, q) for q in pool]
    for q in ids:
        ctx.query(q).close()
    chunk = 1 << 13
    one = gj.NativeServer(ctx, n_slots=1, chunk_rows=chunk)
    alone, _ = one.run(ids, np.arange(len(ids)) * 0.002)
    one.close()
    for r, t in zip(alone, ref):
        assert r["status"] == gj.GJ_OK and r["total"] == t
        assert r["chunk_rows"] == min(chunk, t)
    rng = np.random.default_rng(4)
    picks = rng.integers(0, len(ids), size=400)
    many = gj.NativeServer(ctx, n_slots=8, chunk_rows=chunk)
    mix, stats = many.run([ids[p] for p in picks], np.zeros(400))
    many.close()
    assert stats["peak_in_flight"] > 1
    for r, p in zip(mix, picks):
        a = alone[int(p)]
        assert r["status"] == gj.GJ_OK
        assert (r["total"], r["chunk_rows"], r["chunk_hash"]) == (a["total"], a["chunk_rows"], a["chunk_hash"])
    # admission never exceeds the budget; a request larger than it is refused
    tiny = gj.NativeServer(ctx, n_slots=4, hbm_budget=1, chunk_rows=chunk)
    res, st = tiny.run(ids[:3], [0.0, 0.0, 0.0])
    tiny.close()
    assert all(r["status"] == gj.GJ_ERR_OOM for r in res)
    for q in ids:
        for x in q:
            ctx.release_relation(x)
    ctx.close()
