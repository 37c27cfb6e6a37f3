"""Failure paths on the GPU, made on purpose without faulting or hanging
the device: a bounded wait that runs out (the first tile of the factor
build's group scan never publishes its count; every other tile gives up
after a short poll limit) and device allocations that fail.  Each call
reports its status, and the context stays usable afterwards."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    c = gj.Context(0)
    yield c
    c.close()


def _check_factor(ctx, rid, cols, order, n):
    perm, gstart, gkey = ctx.factor_export(rid, n, len(cols), order)
    ref = np.lexsort([cols[c] for c in reversed(order)])
    assert np.array_equal(perm.cpu().numpy(), ref)
    srt = np.stack([cols[c][ref] for c in range(len(cols))], axis=1)
    head = np.ones(n, bool)
    head[1:] = (srt[1:] != srt[:-1]).any(axis=1)
    assert np.array_equal(gstart.cpu().numpy()[:-1], np.flatnonzero(head))
    assert np.array_equal(gkey.cpu().numpy().T, srt[head])


def test_bounded_wait_runs_out_then_the_context_recovers(ctx):
    from paper_2206_10435_gb300 import gj
    rng = np.random.default_rng(5)
    n = 100_000   # 25 tiles of the group scan: 24 of them wait on the first
    cols = [rng.integers(0, 5000, n, dtype=np.int32), rng.integers(-300, 300, n, dtype=np.int32)]
    rid = ctx.load_relation([torch.from_numpy(c).cuda() for c in cols], [0, 1])
    ctx.set_option(gj.GJ_OPT_SPIN_LIMIT, 2000)
    ctx.set_option(gj.GJ_OPT_TEST_STALL, 1)
    for _ in range(2):
        with pytest.raises(gj.GJError) as e:
            ctx.factor_export(rid, n, 2, [0, 1])
        assert e.value.status == gj.GJ_ERR_TIMEOUT
    ctx.set_option(gj.GJ_OPT_TEST_STALL, 0)
    ctx.set_option(gj.GJ_OPT_SPIN_LIMIT, 0)
    _check_factor(ctx, rid, cols, [0, 1], n)
    _check_factor(ctx, rid, cols, [1, 0], n)
    ctx.release_relation(rid)
    # a whole query afterwards: the same result as the oracle's
    q = G.chain3_uniform(seed=17, rows=3000, end_domain=500, mid_domain=60)
    ids = gj.load_query(ctx, q)
    qq = ctx.query(ids)
    total = qq.summarize()
    ref = O.join(q)
    assert total == ref.rowids.shape[0]
    cols_out, rids = qq.desummarize(0, total, rowids=True)
    got = np.stack([r.cpu().numpy() for r in rids], axis=1)
    assert np.array_equal(got, ref.rowids)
    qq.close()
    for i in ids:
        ctx.release_relation(i)


def test_invalid_failure_options_are_rejected(ctx):
    from paper_2206_10435_gb300 import gj
    for opt, bad in ((gj.GJ_OPT_SPIN_LIMIT, -1), (gj.GJ_OPT_SPIN_LIMIT, 1 << 23),
                     (gj.GJ_OPT_TEST_STALL, 2), (gj.GJ_OPT_FAIL_ALLOC_AT, -3)):
        with pytest.raises(gj.GJError) as e:
            ctx.set_option(opt, bad)
        assert e.value.status == gj.GJ_ERR_INVALID


def test_failed_allocations_report_oom_and_leak_nothing(ctx):
    """Every device allocation of a whole pipeline (factors, summary, a
    desummarised window with row ids, a GFJS level) made to fail in turn:
    each run reports GJ_ERR_OOM, and once the query and relations are gone
    the context's pool holds exactly what it held before.  A clean run
    afterwards gives the oracle's rows."""
    from paper_2206_10435_gb300 import gj
    q = G.chain3_uniform(seed=23, rows=2000, end_domain=300, mid_domain=40)
    ref = O.join(q)

    def pipeline():
        ids = gj.load_query(ctx, q)
        try:
            qq = ctx.query(ids)
            try:
                total = qq.summarize()
                _, rids = qq.desummarize(0, total, rowids=True)
                qq.level(1, 0, total)
                torch.cuda.synchronize()
                return total, np.stack([r.cpu().numpy() for r in rids], axis=1)
            finally:
                qq.close()
        finally:
            for i in ids:
                ctx.release_relation(i)

    base, _ = ctx.pool_usage()
    ctx.set_option(gj.GJ_OPT_FAIL_ALLOC_AT, 1 << 40)   # count them, fail none
    pipeline()
    _, n_allocs = ctx.pool_usage()
    assert n_allocs > 20
    for n in range(1, n_allocs + 1):
        ctx.set_option(gj.GJ_OPT_FAIL_ALLOC_AT, n)
        with pytest.raises(gj.GJError) as e:
            pipeline()
        assert e.value.status == gj.GJ_ERR_OOM, (n, e.value.status)
        ctx.set_option(gj.GJ_OPT_FAIL_ALLOC_AT, 0)
        used, _ = ctx.pool_usage()
        assert used == base, (n, used, base)
    total, rids = pipeline()
    assert total == ref.rowids.shape[0]
    assert np.array_equal(rids, ref.rowids)
