"""The cyclic 3-way join R(A,B) |><| S(B,C) |><| T(C,A) on the GPU against
the oracle: |Q|, every row (row ids and columns) in canonical order, windows
across emit tiles, the empty result, 2^64 overflow, and the calls that have
no meaning for its cluster summary.  Every case runs with each way of
intersecting the segments (chosen, sorted lists, bitmaps).  Integer work:
exact equality."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests.gpu_util import Run
from tests.test_oracle import _paper_triangle, tiny_triangles

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1, 2], ids=["chosen", "lists", "bitmaps"])
def ctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    c = gj.Context(0)
    c.set_option(gj.GJ_OPT_TRIANGLE_INTERSECT, request.param)
    yield c
    c.close()


def triangle_parity(ctx, q, windows=()):
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


def test_paper_example(ctx):
    # Section 3.2.1: entries (a1,b1,5), (b1,c1,10), (c1,a1,20) -> (a1,b1,c1,1000)
    assert triangle_parity(ctx, _paper_triangle(), windows=[(999, 5)]) == 1010


@pytest.mark.parametrize("i", range(60))
def test_tiny_triangles(ctx, i):
    triangle_parity(ctx, tiny_triangles()[i], windows=[(0, 1), (1, 2), (2, 5)])


@pytest.mark.parametrize("seed,s", [(0, 0.0), (1, 0.8), (2, 1.2)])
def test_several_tiles(ctx, seed, s):
    q = G.triangle_query(300 + seed, [2000, 1500, 2500], domain=40, s=s)
    total = triangle_parity(ctx, q, windows=[(0, 5000), (1023, 4099), (7777, 3000)])
    assert total > 5000


def test_larger_with_windows(ctx):
    q = G.triangle_query(41, [20_000, 20_000, 20_000], domain=300, s=0.7, payload_dtype=np.int32)
    total = triangle_parity(ctx, q, windows=[(123_457, 200_000)])
    assert total > 200_000


def test_no_triangle_closes(ctx):
    # A takes even values in R and odd values in T: nothing closes the cycle
    q = G.triangle_query(5, [50, 50, 50], domain=10)
    R, T = q.relations[0], q.relations[2]
    R.keys[0] = (R.keys[0] * 2).astype(np.int32)
    T.keys[1] = (T.keys[1] * 2 + 1).astype(np.int32)
    assert triangle_parity(ctx, q) == 0


def test_overflow_reported(ctx):
    # all keys equal: |Q| = 2^22 * 2^22 * 2^22 > 2^64
    from paper_2206_10435_gb300 import gj
    n = 1 << 22
    rels = [G.Relation(nm, at, [np.zeros(n, np.int32)] * 2) for nm, at in
            (("R", [0, 1]), ("S", [1, 2]), ("T", [2, 0]))]
    q = G.Query("tri_overflow", rels, {0: "A", 1: "B", 2: "C"})
    ids = gj.load_query(ctx, q)
    qq = ctx.query(ids)
    with pytest.raises(gj.GJError) as e:
        qq.summarize()
    assert e.value.status == gj.GJ_ERR_OVERFLOW
    qq.close()
    for x in ids:
        ctx.release_relation(x)


def test_tree_only_calls_rejected(ctx):
    from paper_2206_10435_gb300 import gj
    q = G.triangle_query(9, [30, 30, 30], domain=5)
    run = Run(ctx, q)
    assert run.summarize() > 0
    with pytest.raises(gj.GJError) as e:
        run.q.level(0, 0, 10)
    assert e.value.status == gj.GJ_ERR_INVALID
    with pytest.raises(gj.GJError) as e:
        run.q.summary_groups(0)
    assert e.value.status == gj.GJ_ERR_INVALID
    run.close()


@pytest.mark.parametrize("shift", [-2**31, -17, 2**31 - 64])
def test_keys_at_the_int32_ends(ctx, shift):
    # bitmap rows and bits are offsets from the smallest key: keys next to
    # INT32_MIN / INT32_MAX must not wrap
    q = G.triangle_query(77, [400, 300, 500], domain=60, s=0.5)
    for r in q.relations:
        r.keys = [(k.astype(np.int64) + shift).astype(np.int32) for k in r.keys]
    assert triangle_parity(ctx, q, windows=[(5, 900)]) > 0


def test_c_ranges_of_s_and_t_differ(ctx):
    # S's c values in [0, 40), T's in [25, 90): only [25, 40) can close the cycle
    q = G.triangle_query(78, [300, 400, 400], domain=40)
    T = q.relations[2]
    T.keys[0] = (T.keys[0] * 65 // 40 + 25).astype(np.int32)
    assert triangle_parity(ctx, q, windows=[(3, 100)]) > 0


def test_c_range_too_wide_for_bitmaps(ctx):
    # C spans all of int32: bitmaps would take 2^29 bytes per row, so every
    # mode intersects sorted lists; the result is the same
    q = G.triangle_query(79, [200, 200, 200], domain=8)
    S, T = q.relations[1], q.relations[2]
    S.keys[1] = np.where(S.keys[1] == 0, np.int32(-2**31), S.keys[1]).astype(np.int32)
    T.keys[0] = np.where(T.keys[0] == 7, np.int32(2**31 - 1), T.keys[0]).astype(np.int32)
    assert triangle_parity(ctx, q) > 0


def test_intersect_option_validated(ctx):
    from paper_2206_10435_gb300 import gj
    for bad in (-1, 3):
        with pytest.raises(gj.GJError) as e:
            ctx.set_option(gj.GJ_OPT_TRIANGLE_INTERSECT, bad)
        assert e.value.status == gj.GJ_ERR_INVALID
