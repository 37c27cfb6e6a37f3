"""The downward pass's ways of adding contributions to a child's down message
(GJ_OPT_DOWN_COMBINE: combined per block where the links are out of key
order, never, always) all give the oracle's summary -- |Q|, every key
tuple's multiplicity, the rows -- on skewed chains (hot keys), a star whose
leading-column child has long runs of equal keys, and random trees; the
summary autotuner times them and keeps one.  Integer sums: exact equality."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests.gpu_util import Run, to_u64
from tests.test_gpu_parity import full_parity

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


def _queries():
    return [
        G.chain5_zipf(rows=30_000, domain=5_000, s=1.1),       # 7.6e6 rows, hot keys
        G.chain5_zipf(rows=30_000, domain=20_000, s=0.0),      # 1.5e5 rows
        G.star_poisson(seed=11, fact_rows=40_000, domain=3_000, n_dims=4, lam=2.0),
        G.random_tree_query(4321, 5, max_rows=200, domain=20, max_new=2, min_rows=50),
    ]


@pytest.mark.parametrize("qi", range(4))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_every_mode_gives_the_oracle_summary(ctx, qi, mode):
    from paper_2206_10435_gb300 import gj
    ctx.set_option(gj.GJ_OPT_DOWN_COMBINE, mode)
    q = _queries()[qi]
    full_parity(ctx, q, check_levels=False, windows=[(0, 1), (777, 3000)])


def test_modes_agree_group_by_group(ctx):
    from paper_2206_10435_gb300 import gj
    q = G.chain5_zipf(rows=200_000, domain=50_000, s=1.1)
    tables = []
    for mode in (0, 1, 2):
        ctx.set_option(gj.GJ_OPT_DOWN_COMBINE, mode)
        run = Run(ctx, q)
        run.summarize()
        tabs = []
        for rel in range(len(q.relations)):
            w, m, o = run.q.summary_groups(rel)
            tabs.append((to_u64(w), to_u64(m), to_u64(o)))
        tables.append(tabs)
        run.close()
    for t in tables[1:]:
        for (w0, m0, o0), (w1, m1, o1) in zip(tables[0], t):
            assert np.array_equal(w0, w1) and np.array_equal(m0, m1) and np.array_equal(o0, o1)


def test_invalid_values_rejected(ctx):
    from paper_2206_10435_gb300 import gj
    for bad in (-1, 3):
        with pytest.raises(gj.GJError) as e:
            ctx.set_option(gj.GJ_OPT_DOWN_COMBINE, bad)
        assert e.value.status == gj.GJ_ERR_INVALID


def test_summary_autotuner(ctx, tmp_path):
    from paper_2206_10435_gb300 import autotune, gj
    q = G.chain5_zipf(rows=50_000, domain=10_000, s=1.1)
    run = Run(ctx, q)
    cache = str(tmp_path / "tune.json")
    first = autotune.tune_summary(ctx, run.q, reps=1, cache_path=cache)
    assert first["down_combine"] in (0, 1, 2) and not first["cached"]
    assert set(first["candidates_ms"]) == {"0", "1", "2"}
    again = autotune.tune_summary(ctx, run.q, reps=1, cache_path=cache)
    assert again["cached"] and again["down_combine"] == first["down_combine"]
    assert run.summarize() == O.count(q).total
    run.close()
    # the 3-cycle: its intersection choice
    tq = G.triangle_query(77, [3000, 2500, 2000], domain=60, s=0.5)
    trun = Run(ctx, tq)
    t = autotune.tune_summary(ctx, trun.q, triangle=True, reps=1, cache_path=cache)
    assert t["triangle_intersect"] in (1, 2)
    assert trun.summarize() == O.count(tq).total
    trun.close()
    ctx.set_option(gj.GJ_OPT_DOWN_COMBINE, 0)
    ctx.set_option(gj.GJ_OPT_TRIANGLE_INTERSECT, 0)
