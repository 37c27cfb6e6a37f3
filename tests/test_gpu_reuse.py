"""Compute-and-reuse: a stored summary, loaded without the original
relations, desummarises to exactly the same rows, levels and per-group
multiplicities (and those equal the oracle's)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests import golden_fig
from tests.gpu_util import to_u64

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


def _queries():
    fig, *_ = golden_fig.load()
    return [fig, G.chain3_uniform(rows=3000, end_domain=2000, mid_domain=200),
            G.star_poisson(fact_rows=20_000, domain=5000),
            G.random_tree_query(77, 4, max_rows=40, domain=5, max_new=2, min_rows=20, max_shared=2),
            G.chain5_zipf(rows=20_000, domain=20_000)]


@pytest.mark.parametrize("qi", range(5))
def test_saved_summary_reproduces_the_result(ctx, tmp_path, qi):
    from paper_2206_10435_gb300 import gj
    q = _queries()[qi]
    ids = gj.load_query(ctx, q)
    qq = ctx.query(ids)
    total = qq.summarize()
    cols, rids = qq.desummarize(0, total, rowids=True)
    cols = [c.cpu().numpy() for c in cols]
    levels = [tuple(t.cpu().numpy() for t in qq.level(l, 0, total)) for l in range(len(qq.var_attr))]
    groups = [tuple(to_u64(t) for t in qq.summary_groups(r)) for r in range(qq.n_rel)]
    path = os.path.join(tmp_path, "summary.gjs")
    nbytes = qq.save(path)
    assert nbytes == os.path.getsize(path)
    qq.close()
    for r in ids:                      # the originals are gone
        ctx.release_relation(r)
    lq = gj.Query.load(ctx, path)
    assert lq.total == total == O.count(q).total
    lcols = [c.cpu().numpy() for c in lq.desummarize(0, total)]
    for a, b in zip(lcols, cols):
        assert np.array_equal(a, b)
    ref = O.columns(q, O.join(q).rowids)
    for a, b in zip(lcols, ref):
        assert np.array_equal(a, b)
    for l, (v, f, o) in enumerate(levels):
        lv, lf, lo = (t.cpu().numpy() for t in lq.level(l, 0, total))
        assert np.array_equal(lv, v) and np.array_equal(lf, f) and np.array_equal(lo, o)
    for r in range(lq.n_rel):
        for a, b in zip((to_u64(t) for t in lq.summary_groups(r)), groups[r]):
            assert np.array_equal(a, b)
    lq.close()


def test_truncated_file_is_rejected(ctx, tmp_path):
    from paper_2206_10435_gb300 import gj
    q = G.chain3_uniform(rows=500, end_domain=100, mid_domain=20)
    ids = gj.load_query(ctx, q)
    qq = ctx.query(ids)
    qq.summarize()
    path = os.path.join(tmp_path, "s.gjs")
    n = qq.save(path)
    with open(path, "r+b") as f:
        f.truncate(n // 2)
    with pytest.raises(gj.GJError) as e:
        gj.Query.load(ctx, path)
    assert e.value.status == gj.GJ_ERR_INVALID
    qq.close()
    for r in ids:
        ctx.release_relation(r)
