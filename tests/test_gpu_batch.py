"""Batched summaries (gj_batch_*) against the oracle and against the
one-query-at-a-time API, bit for bit, with and without a CUDA graph."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CAP = (1 << 64) - 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    c = gj.Context(0)
    yield c
    c.close()


def _special_queries():
    qs = []
    z = lambda n, v=0: np.full(n, v, np.int32)
    # 256^9 = 2^72 ways: overflow
    qs.append(G.Query("over", [G.Relation(f"R{i}", [i, i + 1], [z(256), z(256)]) for i in range(9)]))
    # a dead branch above 2^64 ways
    rels = [G.Relation("R0", [0, 1], [z(3, 1), z(3, 5)]), G.Relation("R1", [1, 2], [z(4, 6), z(4)])]
    rels += [G.Relation(f"R{i}", [i, i + 1], [z(256), z(256)]) for i in range(2, 10)]
    qs.append(G.Query("dead", rels))
    # single relation, and a query with an empty table
    qs.append(G.Query("single", [G.Relation("S", [0, 1], [np.arange(7, dtype=np.int32), z(7)])]))
    e = G.chain_query("empty", [50, 40, 30], [5, 5, 5, 5], [0.5] * 4, None, 3)
    e.relations[1] = G.Relation("R2", [1, 2], [np.zeros(0, np.int32)] * 2)
    qs.append(e)
    # one-key relations (a star with single-attribute children)
    qs.append(G.Query("star1", [G.Relation("F", [0, 1], [np.array([1, 1, 2, 3], np.int32),
                                                          np.array([4, 4, 5, 6], np.int32)]),
                                G.Relation("D0", [0], [np.array([1, 1, 2], np.int32)]),
                                G.Relation("D1", [1], [np.array([4, 6, 6, 6], np.int32)])]))
    return qs


def _load(ctx, queries):
    from paper_2206_10435_gb300 import gj
    return [gj.load_query(ctx, q) for q in queries]


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_matches_oracle_and_plain(ctx, seed):
    from paper_2206_10435_gb300 import gj
    queries = G.batch_queries(seed=100 + seed, n_queries=96, rows_range=(1, 3000),
                              domain_range=(2, 400)) + _special_queries()
    ids = _load(ctx, queries)
    ref = [O.count(q) for q in queries]
    b = gj.Batch(ctx, ids)
    for use_graph in (False, True, True):
        b.totals.zero_()
        b.run(use_graph=use_graph)
        torch.cuda.synchronize()
        tot = b.totals.cpu().numpy().view(np.uint64)
        st = b.status.cpu().numpy()
        for qi, r in enumerate(ref):
            assert int(tot[qi]) == r.total, (qi, queries[qi].name)
            assert st[qi] == (gj.GJ_ERR_OVERFLOW if r.overflow else gj.GJ_OK)
    # the one-query-at-a-time path agrees
    for qi, q in enumerate(ids):
        qq = ctx.query(q)
        try:
            t = qq.summarize()
        except gj.GJError as e:
            assert e.status == gj.GJ_ERR_OVERFLOW and ref[qi].overflow
            t = CAP
        assert t == ref[qi].total
        qq.close()
    b.close()
    for q in ids:
        for r in q:
            ctx.release_relation(r)


def test_batch_grid_sizes_agree(ctx):
    from paper_2206_10435_gb300 import gj
    queries = G.batch_queries(seed=7, n_queries=40, rows_range=(100, 20000),
                              domain_range=(10, 2000))
    ids = _load(ctx, queries)
    ref = [O.count(q).total for q in queries]
    b = gj.Batch(ctx, ids)
    for m in (1, 3, 8):
        b.set_grid_mult(m)
        b.run(use_graph=True)
        torch.cuda.synchronize()
        assert [int(x) for x in b.totals.cpu().numpy().view(np.uint64)] == ref
    b.close()
    for q in ids:
        for r in q:
            ctx.release_relation(r)


def _other_shape_queries():
    """Queries outside the batched kernels' shapes: three-key relations, a
    separator of two attributes, a relation with six children."""
    rng = np.random.default_rng(12)
    r = lambda n, d: rng.integers(0, d, n, dtype=np.int32)
    qs = []
    # a three-key root with two children
    qs.append(G.Query("three", [G.Relation("F", [0, 1, 2], [r(300, 6), r(300, 5), r(300, 7)]),
                                G.Relation("A", [0, 3], [r(40, 6), r(40, 4)]),
                                G.Relation("B", [2], [r(30, 7)])]))
    # a child joined on two attributes
    qs.append(G.Query("twosep", [G.Relation("P", [0, 1], [r(200, 4), r(200, 5)]),
                                 G.Relation("C", [0, 1, 2], [r(150, 4), r(150, 5), r(150, 9)]),
                                 G.Relation("D", [2], [r(20, 9)])]))
    # six children of one relation (the batched kernels take up to 16)
    qs.append(G.Query("six", [G.Relation("H", [0], [r(50, 8)])] +
                      [G.Relation(f"K{i}", [0, 10 + i], [r(30, 8), r(30, 3)]) for i in range(6)]))
    # three-key relations all through a chain
    qs.append(G.Query("wide3", [G.Relation("X", [0, 1, 2], [r(100, 3), r(100, 3), r(100, 4)]),
                                G.Relation("Y", [2, 3, 4], [r(100, 4), r(100, 3), r(100, 3)])]))
    # cyclic queries: a 4-cycle and two triangles sharing an edge
    qs.append(G.cyclic_query(5, "square", 60, domain=5))
    qs.append(G.cyclic_query(6, "diamond", 40, domain=4))
    return qs


def test_batch_takes_every_acyclic_shape(ctx):
    """Chains the batched kernels take, mixed with queries they do not (the
    batch summarises those through the single-query path): every total and
    status equals the oracle's, with and without the graph, and a batch of
    only such queries works too."""
    from paper_2206_10435_gb300 import gj
    others = _other_shape_queries()
    queries = G.batch_queries(seed=44, n_queries=30, rows_range=(1, 2000), domain_range=(2, 300))
    mixed = []
    for i, q in enumerate(queries):
        mixed.append(q)
        if i % 8 == 3:
            mixed.append(others[(i // 8) % len(others)])
    mixed += others
    for qs in (mixed, others):
        ids = _load(ctx, qs)
        ref = [O.count(q) for q in qs]
        b = gj.Batch(ctx, ids)
        # the six-children query is batched; the others take the single-query path
        single = [o for o in others if o.name != "six"]
        batched = [q for q in qs if all(q is not o for o in single)]
        assert b.n_relations == sum(len(q.relations) for q in batched)
        for use_graph in (False, True, True):
            b.run(use_graph=use_graph)
            torch.cuda.synchronize()
            tot = b.totals.cpu().numpy().view(np.uint64)
            st = b.status.cpu().numpy()
            for j, c in enumerate(ref):
                assert int(tot[j]) == (CAP if c.overflow else c.total), (j, qs[j].name)
                assert st[j] == (gj.GJ_ERR_OVERFLOW if c.overflow else gj.GJ_OK), j
        b.close()
        for q in ids:
            for x in q:
                ctx.release_relation(x)


def test_batch_rejects_a_cross_product(ctx):
    from paper_2206_10435_gb300 import gj
    a = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    r0 = ctx.load_relation([a, a], [0, 1])
    r1 = ctx.load_relation([a, a], [2, 3])
    with pytest.raises(gj.GJError) as e:
        gj.Batch(ctx, [[r0, r1]])
    assert e.value.status == gj.GJ_ERR_INVALID
    for r in (r0, r1):
        ctx.release_relation(r)
