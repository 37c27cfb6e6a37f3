"""Early projection (Section 3.7) on the GPU against the oracle: attributes
held by one relation are deleted before the summary is built; the result is
the same bag of row-id tuples, without those columns, ordered by the
remaining variables and then the row ids.  Integer work: exact equality."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests.gpu_util import Run, to_u64
from tests.test_oracle import droppable, tiny_queries

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


def projected_parity(ctx, q, drop, windows=()):
    run = Run(ctx, q, drop)
    total = run.summarize()
    assert total == O.count(q).total
    if total:
        j = O.join(q, drop=drop)
        ref = O.columns(q, j.rowids, drop)
        cols, rids = run.rows()
        assert len(cols) == len(ref)
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
        lv = O.gfjs_levels(q, j.rowids, drop)
        for l in range(len(lv)):
            val, freq, off = run.q.level(l, 0, total)
            assert np.array_equal(val.cpu().numpy(), lv[l].value)
            assert np.array_equal(to_u64(freq), lv[l].freq)
            assert np.array_equal(to_u64(off), lv[l].offset)
    # the relation that held a dropped attribute groups by fewer columns
    for rel, R in enumerate(q.relations):
        keep = [c for c, a in enumerate(R.attrs) if a not in drop]
        if R.n_rows and len(keep) < len(R.attrs):
            distinct = np.unique(np.stack([R.keys[c] for c in keep], axis=1), axis=0).shape[0]
            assert run.q.n_groups[rel] == distinct
    run.close()
    return total


@pytest.mark.parametrize("q", [q for q in tiny_queries() if droppable(q)][:60],
                         ids=lambda q: q.name)
def test_tiny_trees(ctx, q):
    cand = droppable(q)
    projected_parity(ctx, q, cand[:1], windows=[(0, 1), (1, 2)])
    projected_parity(ctx, q, cand, windows=[(3, 5)])


@pytest.mark.parametrize("seed", range(8))
def test_several_tiles(ctx, seed):
    q = G.random_tree_query(1000 + seed, 2 + seed % 4, max_rows=60, domain=6, max_new=2,
                            min_rows=20)
    cand = droppable(q)
    if not cand:
        pytest.skip("no attribute held by one relation")
    projected_parity(ctx, q, cand, windows=[(0, 5000), (1023, 4099)])


def test_chain5_zipf_ends_dropped(ctx):
    # K0 and K5 are held by R1 and R5 only
    q = G.chain5_zipf(rows=20_000, domain=20_000)
    total = projected_parity(ctx, q, [0, 5], windows=[(12345, 100_000)])
    assert total > 0


def test_shared_attribute_rejected(ctx):
    from paper_2206_10435_gb300 import gj
    q = G.chain5_zipf(rows=1000, domain=1000)
    ids = gj.load_query(ctx, q)
    for bad in ([1], [9]):          # K1 joins R1 and R2; attribute 9 is held by nobody
        with pytest.raises(gj.GJError) as ei:
            ctx.query(ids, drop_attrs=bad)
        assert ei.value.status == gj.GJ_ERR_INVALID
    for i in ids:
        ctx.release_relation(i)
