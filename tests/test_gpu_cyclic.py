"""General cyclic queries on the GPU (one-maxclique junction tree, built
at group level relation by relation) against the oracle's plain
definition: |Q|, every row (row ids and columns) in canonical order over V
by first appearance, windows across emit tiles, the empty result, 2^64
overflow, and the calls with no meaning for a cyclic summary.  Integer
work: exact equality."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests.gpu_util import Run
from tests.test_oracle import tiny_cyclic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    c = gj.Context(0)
    yield c
    c.close()


def cyclic_parity(ctx, q, windows=()):
    run = Run(ctx, q)
    total = run.summarize()
    assert total == O.count(q).total
    if total:
        j = O.join(q)
        ref = O.columns(q, j.rowids)
        cols, rids = run.rows()
        assert np.array_equal(rids, j.rowids)
        for a, b in zip(cols, ref):
            assert np.array_equal(a, b)
        for r0, n in windows:
            if r0 >= total:
                continue
            cw, rw = run.rows(r0, n)
            m = min(n, total - r0)
            assert np.array_equal(rw, j.rowids[r0:r0 + m])
            for a, b in zip(cw, ref):
                assert np.array_equal(a, b[r0:r0 + m])
    run.close()
    return total


TINY = tiny_cyclic()


@pytest.mark.parametrize("i", range(len(TINY)))
def test_tiny_cyclic_queries(ctx, i):
    cyclic_parity(ctx, TINY[i])


# (rows of the first relation, key domain): results of 10^4 .. 2.1 x 10^5 rows
SIZES = {"square": (300, 24), "pentagon": (120, 12), "bowtie": (50, 8), "diamond": (110, 10),
         "k4": (60, 8), "wide": (300, 6), "pendant": (70, 10)}


@pytest.mark.parametrize("shape", list(G.CYCLIC_SHAPES))
def test_every_shape_across_emit_tiles(ctx, shape):
    k = len(G.CYCLIC_SHAPES[shape])
    base, dom = SIZES[shape]
    rows = [base + 13 * i for i in range(k)]
    total = cyclic_parity(ctx, G.cyclic_query(8100 + k, shape, rows, domain=dom, s=0.6),
                          windows=[(0, 1), (3, 1500), (1023, 4097), (9000, 777)])
    assert total > 4096


def test_empty_result(ctx):
    # S's B values never meet R's
    q = G.cyclic_query(3, "square", 50, domain=6)
    q.relations[1].keys[0] = (q.relations[1].keys[0] + 100).astype(np.int32)
    assert cyclic_parity(ctx, q) == 0


def test_overflow_reported(ctx):
    from paper_2206_10435_gb300 import gj
    # a 4-cycle of identical keys: 2^16 rows per relation gives 2^64 rows
    z = lambda n: np.zeros(n, np.int32)
    rels = [G.Relation(f"R{i}", list(at), [z(1 << 16), z(1 << 16)])
            for i, at in enumerate(G.CYCLIC_SHAPES["square"])]
    run = Run(ctx, G.Query("sq_over", rels))
    with pytest.raises(gj.GJError) as e:
        run.summarize()
    assert e.value.status == gj.GJ_ERR_OVERFLOW
    run.close()
    # one row fewer in one relation: 2^64 - 2^48, exact
    rels[0] = G.Relation("R0", [0, 1], [z((1 << 16) - 1), z((1 << 16) - 1)])
    run = Run(ctx, G.Query("sq_exact", rels))
    assert run.summarize() == ((1 << 16) - 1) << 48
    run.close()


@pytest.mark.parametrize("shape", ["triangle", "square"])
def test_window_contract(ctx, shape):
    """The desummarise windows of the two cyclic paths (the 3-cycle's and
    the junction tree's): GJ_ERR_STATE before the summary, empty windows and
    windows at or past |Q| write nothing, a window reaching past |Q| is
    clipped, a clipped window of 2^31 rows is refused, and rows past 2^32 of
    one huge block (all keys equal: n^k rows, row r the row-id tuple of r's
    base-n digits) are exact."""
    from paper_2206_10435_gb300 import gj
    tri = shape == "triangle"
    attrs = [(0, 1), (1, 2), (2, 0)] if tri else G.CYCLIC_SHAPES["square"]
    q = G.triangle_query(77, [300, 250, 200], domain=20) if tri else \
        G.cyclic_query(31, "square", 120, domain=10)
    run = Run(ctx, q)
    with pytest.raises(gj.GJError) as e:
        run.q.desummarize(0, 4)
    assert e.value.status == gj.GJ_ERR_STATE
    total = run.summarize()
    assert total == O.count(q).total > 3
    j = O.join(q)
    ref = O.columns(q, j.rowids)
    for r0, n in [(0, 0), (total, 5), (1 << 63, 5)]:
        assert all(c.numel() == 0 for c in run.q.desummarize(r0, n))
    cols = run.q.desummarize(total - 3, (1 << 64) - 1, out=run.q.alloc_columns(3))
    for a, b in zip(cols, ref):
        assert np.array_equal(a.cpu().numpy(), b[total - 3:])
    run.close()
    n, k = (2000, 3) if tri else (300, 4)
    eq = G.Query(shape + "_equal", [G.Relation(f"R{i}", list(at), [np.full(n, 7, np.int32) for _ in at])
                                    for i, at in enumerate(attrs)])
    run = Run(ctx, eq)
    assert run.summarize() == n ** k
    with pytest.raises(gj.GJError) as e:
        run.q.desummarize(5, 1 << 31, out=run.q.alloc_columns(1))
    assert e.value.status == gj.GJ_ERR_INVALID
    r0 = (1 << 32) + 5
    cols, rids = run.q.desummarize(r0, 2, out=run.q.alloc_columns(2), rowids=True)
    assert [c.cpu().tolist() for c in cols] == [[7, 7]] * len(cols)
    for i, r in enumerate((r0, r0 + 1)):
        assert [int(t[i]) for t in rids] == [r // n ** (k - 1 - p) % n for p in range(k)]
    run.close()


def test_tree_only_calls_rejected(ctx):
    from paper_2206_10435_gb300 import gj
    run = Run(ctx, G.cyclic_query(9, "square", 30, domain=4))
    assert run.summarize() > 0
    for call in (lambda: run.q.level(0, 0, 10), lambda: run.q.summary_groups(0)):
        with pytest.raises(gj.GJError) as e:
            call()
        assert e.value.status == gj.GJ_ERR_INVALID
    run.close()


@pytest.mark.parametrize("spread", [1, -7, 1000003])
def test_key_ranges_wide_narrow_and_negative(ctx, spread):
    """The count step narrows its searches through a table over the first
    shared column's value range when that range is small next to the groups;
    keys stretched far apart (no table) or shifted negative give the same
    rows as the oracle."""
    q = G.cyclic_query(8200 + abs(spread) % 97, "pentagon", [220, 240, 260, 280, 300], domain=11, s=0.4)
    for R in q.relations:
        R.keys[:] = [(k.astype(np.int64) * spread - (5 if spread < 0 else 0)).astype(np.int32) for k in R.keys]
    assert cyclic_parity(ctx, q, windows=[(5, 999)]) > 0


@pytest.mark.parametrize("flip", [False, True])
def test_two_cliques_and_one(ctx, flip):
    """A 4-cycle is answered on two maxcliques ({A,B,C} and {C,D,A}, joined
    on {A,C}) whichever way its last relation's columns are declared (its
    factor is ordered by D, the column it shares with R2, first); the rows
    are the oracle's either way."""
    q = G.cyclic_query(8400, "square", [700, 650, 600, 550], domain=40, s=0.7)
    if flip:
        R = q.relations[3]
        q.relations[3] = G.Relation(R.name, R.attrs[::-1], R.keys[::-1], R.payloads)
    assert cyclic_parity(ctx, q, windows=[(0, 4097), (12345, 777)]) > 4096
