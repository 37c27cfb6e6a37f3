"""The native serving runtime (gj_server_*): join sizes against the oracle,
and every request's streamed result (all its chunks, by their hash)
identical when the request runs alone and when it runs mixed with
concurrent requests; the hash of a request's rows equals the hash of the
oracle's result columns."""
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


def _mix64(x):
    M = (1 << 64) - 1
    x ^= x >> 30
    x = (x * 0xbf58476d1ce4e5b9) & M
    x ^= x >> 27
    x = (x * 0x94d049bb133111eb) & M
    x ^= x >> 31
    return x


def _hash_columns(cols):
    """The server's hash of result rows 0..n-1: xor over columns c and rows i
    of mix(v ^ mix(c << 40 ^ i)), v the value as an unsigned 32/64-bit word."""
    h = 0
    for c, col in enumerate(cols):
        bits = 32 if col.dtype.itemsize == 4 else 64
        for i, v in enumerate(col.tolist()):
            h ^= _mix64((int(v) & ((1 << bits) - 1)) ^ _mix64((c << 40) ^ i))
    return h


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
    limit = 5 * chunk + 17         # several chunks and a ragged last one
    one = gj.NativeServer(ctx, n_slots=1, chunk_rows=chunk, max_rows=limit)
    alone, _ = one.run(ids, np.arange(len(ids)) * 0.002)
    one.close()
    for r, t in zip(alone, ref):
        assert r["status"] == gj.GJ_OK and r["total"] == t
        assert r["rows"] == min(limit, t)
        assert r["t_last"] >= r["t_chunk"] >= r["t_summary"] >= r["t_arrival"]
    # the hash of the streamed rows is the hash of the oracle's columns
    for q, r in list(zip(pool, alone))[:6]:
        j = O.join(q)
        cols = O.columns(q, j.rowids[:r["rows"]])
        assert r["hash"] == _hash_columns(cols)
    rng = np.random.default_rng(4)
    picks = rng.integers(0, len(ids), size=400)
    many = gj.NativeServer(ctx, n_slots=8, chunk_rows=chunk, max_rows=limit)
    mix, stats = many.run([ids[p] for p in picks], np.zeros(400))
    many.close()
    assert stats["peak_in_flight"] > 1
    for r, p in zip(mix, picks):
        a = alone[int(p)]
        assert r["status"] == gj.GJ_OK
        assert (r["total"], r["rows"], r["hash"]) == (a["total"], a["rows"], a["hash"])
    # admission never exceeds the budget; a request larger than it is refused
    tiny = gj.NativeServer(ctx, n_slots=4, hbm_budget=1, chunk_rows=chunk)
    res, st = tiny.run(ids[:3], [0.0, 0.0, 0.0])
    tiny.close()
    assert all(r["status"] == gj.GJ_ERR_OOM for r in res)
    for q in ids:
        for x in q:
            ctx.release_relation(x)
    ctx.close()


def _small_pool(n=8, seed=19):
    """Chains of 2-4 tables with results of 10^2..3*10^4 rows (the oracle
    materialises them whole)."""
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        k = int(rng.integers(2, 5))
        rows = rng.integers(50, 800, size=k)
        doms = rng.integers(20, 300, size=k + 1)
        s = float(rng.uniform(0, 1.2))
        qs.append(G.chain_query(f"a{i}", rows, doms, [s] * (k + 1), np.int64 if i % 2 else np.int32,
                                3000 + i))
    return qs


@pytest.mark.parametrize("arena", [0, 1 << 16, 1 << 22])
def test_slot_arena_sizes_give_the_same_results(arena):
    """Each slot takes its requests' device memory from a bump arena: none
    (every allocation from the slot's pool), one too small for any request
    (the summary and every chunk continue in the pool part way), and one
    that holds small requests whole.  Sizes, streamed rows and their hashes
    equal the oracle's, whatever the arena."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    ctx = gj.Context(0, torch.cuda.Stream())
    ctx.set_option(gj.GJ_OPT_SLOT_ARENA, arena)
    pool = _small_pool()
    ref = [O.count(q).total for q in pool]
    ids = [gj.load_query(ctx, q) for q in pool]
    chunk = 1 << 12
    limit = 3 * chunk + 5
    srv = gj.NativeServer(ctx, n_slots=4, chunk_rows=chunk, max_rows=limit)
    picks = [i % len(ids) for i in range(48)]
    res, _ = srv.run([ids[p] for p in picks], np.zeros(len(picks)))
    srv.close()
    hashes = {}
    for q, qi in zip(pool, range(len(pool))):
        j = O.join(q)
        hashes[qi] = _hash_columns(O.columns(q, j.rowids[:min(limit, ref[qi])]))
    for r, p in zip(res, picks):
        assert r["status"] == gj.GJ_OK
        assert r["total"] == ref[p] and r["rows"] == min(limit, ref[p])
        assert r["hash"] == hashes[p]
    for q in ids:
        for x in q:
            ctx.release_relation(x)
    ctx.close()


def test_slot_arena_option_range():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    ctx = gj.Context(0)
    for bad in (-1, (1 << 40) + 1):
        with pytest.raises(gj.GJError) as e:
            ctx.set_option(gj.GJ_OPT_SLOT_ARENA, bad)
        assert e.value.status == gj.GJ_ERR_INVALID
    ctx.close()


def test_server_answers_cyclic_queries():
    """Cyclic queries (a 3-cycle, a 4-cycle on two maxcliques, two triangles
    sharing an edge) served beside trees, with a small slot arena so that
    their intermediate items spill into the pools: sizes and streamed rows
    equal the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    ctx = gj.Context(0, torch.cuda.Stream())
    ctx.set_option(gj.GJ_OPT_SLOT_ARENA, 1 << 20)
    pool = [G.triangle_query(51, [300, 280, 260], domain=25),
            G.cyclic_query(52, "square", [400, 380, 360, 340], domain=30),
            G.cyclic_query(53, "diamond", 150, domain=12)] + _small_pool(n=3, seed=23)
    ref = [O.count(q).total for q in pool]
    ids = [gj.load_query(ctx, q) for q in pool]
    chunk = 1 << 12
    limit = 2 * chunk + 3
    srv = gj.NativeServer(ctx, n_slots=3, chunk_rows=chunk, max_rows=limit)
    picks = [i % len(ids) for i in range(24)]
    res, _ = srv.run([ids[p] for p in picks], np.zeros(len(picks)))
    srv.close()
    hashes = {}
    for qi, q in enumerate(pool):
        j = O.join(q)
        hashes[qi] = _hash_columns(O.columns(q, j.rowids[:min(limit, ref[qi])]))
    for r, p in zip(res, picks):
        assert r["status"] == gj.GJ_OK
        assert r["total"] == ref[p] and r["rows"] == min(limit, ref[p])
        assert r["hash"] == hashes[p]
    for q in ids:
        for x in q:
            ctx.release_relation(x)
    ctx.close()
