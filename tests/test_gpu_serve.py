"""The serving loop on the GPU: every request's answer (join size and first
result chunk) is the same when it runs alone and when it runs mixed with
concurrent requests on other streams."""
import numpy as np
import pytest

from paper_2206_10435_gb300 import datagen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pool(n=24, seed=5):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        k = int(rng.integers(2, 6))
        rows = rng.integers(200, 30000, size=k)
        doms = rng.integers(5, 3000, size=k + 1)
        s = float(rng.uniform(0, 1.4))
        qs.append(G.chain_query(f"p{i}", rows, doms, [s] * (k + 1), np.int64, 1000 + i))
    return qs


def test_results_alone_equal_results_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    from paper_2206_10435_gb300.serve import GJEngine, Request, Server, poisson_arrivals, run_stream
    ctx = gj.Context(0, torch.cuda.Stream())
    pool = _pool()
    ids = [gj.load_query(ctx, q) for q in pool]
    for q in ids:                        # resident factors
        ctx.query(q).close()
    chunk = 1 << 14
    # alone: one slot, one request at a time
    alone = {}
    eng1 = GJEngine(ctx, 1, chunk_rows=chunk, keep_results=True, max_rows=3 * chunk + 5)
    srv1 = Server(eng1, n_slots=1)
    for i, q in enumerate(ids):
        r = Request(i, q)
        srv1.submit(r)
        while r.status == "pending":
            import time
            time.sleep(0.001)
        assert r.status in ("ok", "overflow"), r.status
        alone[i] = (r.total, r.result)
    srv1.drain()
    # mixed: 8 slots, 300 requests arriving much faster than they are served
    rng = np.random.default_rng(9)
    picks = rng.integers(0, len(ids), size=300)
    eng8 = GJEngine(ctx, 8, chunk_rows=chunk, keep_results=True, max_rows=3 * chunk + 5)
    srv8 = Server(eng8, n_slots=8)
    reqs = run_stream(srv8, [ids[p] for p in picks], poisson_arrivals(50000.0, 300, seed=3))
    assert srv8.peak_in_flight > 1
    for r, p in zip(reqs, picks):
        assert r.status in ("ok", "overflow"), r.status
        tot, res = alone[int(p)]
        assert r.total == tot
        if res is None:
            assert r.result is None
        else:
            assert len(r.result) == len(res)
            for a, b in zip(r.result, res):
                assert torch.equal(a, b)
    for q in ids:
        for x in q:
            ctx.release_relation(x)
    ctx.close()
