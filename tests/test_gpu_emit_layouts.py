"""The desummarise emit kernel against the oracle on more output layouts:
one payload column per relation (int32, int64, none, or only on some
relations), 1 and 8 relations, row ids requested or not, windows that cross
emit tiles with ragged tails or start inside a block, and blocks whose row
offsets pass 2^32 (closed form: a block of identical keys is the
mixed-radix count over the relations' rows, Section 3.6)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests.gpu_util import Run
from tests.test_gpu_parity import full_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYOUTS = ["i32", "i64", "none", "some"]


@pytest.fixture(scope="module")
def kctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    c = gj.Context(0)
    yield c
    c.close()


def one_payload(q, which):
    """The query with at most one payload column per relation."""
    rels = []
    for j, R in enumerate(q.relations):
        i32 = [p for p in R.payloads if p.dtype == np.int32][:1]
        i64 = [p for p in R.payloads if p.dtype == np.int64][:1]
        pays = {"i32": i32, "i64": i64, "none": [], "some": i64 if j % 2 == 0 else []}[which]
        rels.append(G.Relation(R.name, R.attrs, R.keys, pays))
    return G.Query(f"{q.name}_{which}", rels, q.attr_names)


@pytest.mark.parametrize("seed", range(40))
def test_tiny_trees(kctx, seed):
    n_rel = 1 + seed % 5
    q = G.random_tree_query(seed, n_rel, max_rows=5 if n_rel <= 3 else 4,
                            domain=3 if n_rel <= 2 else 2, max_new=2,
                            min_rows=0 if seed % 7 == 0 else 1)
    full_parity(kctx, one_payload(q, LAYOUTS[seed % 4]), windows=[(0, 1), (1, 2), (3, 5)])


@pytest.mark.parametrize("seed", range(12))
def test_several_tiles(kctx, seed):
    q = G.random_tree_query(1000 + seed, 2 + seed % 4, max_rows=60, domain=6, max_new=2,
                            min_rows=20)
    full_parity(kctx, one_payload(q, LAYOUTS[seed % 4]),
                windows=[(0, 5000), (1023, 4099), (4095, 1), (6000, 2049)])


@pytest.mark.parametrize("s", [0.0, 1.1, 1.5])
def test_chain5_zipf_windows(kctx, s):
    q = G.chain5_zipf(rows=20_000, domain=20_000, s=s)
    full_parity(kctx, q, check_levels=False,
                windows=[(12345, 100_000), (0, 3 * 2048 + 5), (777, 1)])


@pytest.mark.parametrize("k", [1, 8])
def test_fewest_and_most_relations(kctx, k):
    rows = [3000] if k == 1 else [40] * k
    q = G.chain_query(f"chain{k}", rows, [12] * (k + 1), [0.0] * (k + 1), np.int64, seed=77 + k)
    total = full_parity(kctx, q, check_levels=False, windows=[(5, 2049), (100, 1)])
    assert total > 0


def test_rowids_off_same_columns(kctx):
    q = one_payload(G.random_tree_query(1207, 4, max_rows=60, domain=6, max_new=2,
                                        min_rows=20), "i64")
    run = Run(kctx, q)
    total = run.summarize()
    assert total > 5000
    for r0, n in [(0, total), (2047, 4099)]:
        with_ids, _ = run.q.desummarize(r0, n, rowids=True)
        without = run.q.desummarize(r0, n)
        for a, b in zip(with_ids, without):
            assert torch.equal(a, b)
    run.close()


def _uniform_block_query(k, rows):
    """k relations whose rows all hold the same keys: the result is one
    block, rows ordered by (r_1, ..., r_k) with r_k fastest."""
    rng = np.random.default_rng(4242 + k)
    rels = []
    for j in range(k):
        keys = [np.full(rows, 7 + j, np.int32), np.full(rows, 8 + j, np.int32)]
        pays = [rng.integers(-2**62, 2**62, size=rows, dtype=np.int64)]
        rels.append(G.Relation(f"U{j}", [j, j + 1], keys, pays))
    return G.Query(f"uniform_block_{k}", rels, {j: f"K{j}" for j in range(k + 1)})


@pytest.mark.parametrize("k,rows", [(2, 1 << 17), (3, 1 << 12)])
def test_offsets_past_2_32_inside_one_block(kctx, k, rows):
    q = _uniform_block_query(k, rows)
    run = Run(kctx, q)
    total = run.summarize()
    assert total == rows ** k and total > (1 << 33)
    assert O.count(q).total == total
    for r0, n in [((1 << 33) + 12345, 10_000), (total - 5000, 10_000), ((1 << 32) - 3, 4100)]:
        cols, rids = run.q.desummarize(r0, n, rowids=True)
        m = min(n, total - r0)
        qq = np.arange(r0, r0 + m, dtype=np.uint64)
        want = []
        for j in range(k):
            want.append((qq // np.uint64(rows ** (k - 1 - j))) % np.uint64(rows))
        for j in range(k):
            assert np.array_equal(rids[j].cpu().numpy().astype(np.uint64), want[j]), j
        # V = K0..Kk (constant), then one payload per relation
        for v in range(k + 1):
            assert bool((cols[v] == 7 + v).all()), v
        for j in range(k):
            got = cols[k + 1 + j].cpu().numpy()
            assert np.array_equal(got, q.relations[j].payloads[0][want[j].astype(np.int64)]), j
    run.close()


def test_pinned_host_columns(kctx):
    """Rows written straight into pinned host memory equal the device rows."""
    q = one_payload(G.random_tree_query(1207, 4, max_rows=60, domain=6, max_new=2,
                                        min_rows=20), "i64")
    run = Run(kctx, q)
    total = run.summarize()
    for r0, n in [(0, total), (1023, 4099)]:
        dev_cols, _ = run.q.desummarize(r0, n, rowids=True)
        host = [torch.empty(n, dtype=c.dtype, pin_memory=True) for c in dev_cols]
        got = run.q.desummarize(r0, n, out=host)
        for a, b in zip(dev_cols, got):
            assert not b.is_cuda
            assert torch.equal(a.cpu(), b)
    run.close()


def test_pageable_columns_rejected(kctx):
    from paper_2206_10435_gb300 import gj
    q = one_payload(G.random_tree_query(1207, 4, max_rows=60, domain=6, max_new=2,
                                        min_rows=20), "i64")
    run = Run(kctx, q)
    total = run.summarize()
    dev_cols, _ = run.q.desummarize(0, 10, rowids=True)
    pageable = [torch.empty(10, dtype=c.dtype) for c in dev_cols]
    with pytest.raises(gj.GJError) as ei:
        run.q.desummarize(0, 10, out=pageable)
    assert ei.value.status == gj.GJ_ERR_INVALID
    # the context still works
    again, _ = run.q.desummarize(0, 10, rowids=True)
    for a, b in zip(dev_cols, again):
        assert torch.equal(a, b)
    assert total > 0
    run.close()


def test_pinned_host_columns_from_fresh_threads(kctx):
    """Two host threads that have not used CUDA before desummarise alternate
    windows of two queries (own streams) into pinned host columns."""
    import threading
    q = one_payload(G.random_tree_query(1207, 4, max_rows=60, domain=6, max_new=2,
                                        min_rows=20), "i64")
    run = Run(kctx, q)
    total = run.summarize()
    ref, _ = run.q.desummarize(0, total, rowids=True)
    ref = [c.cpu() for c in ref]
    qs = [kctx.query(run.ids) for _ in range(2)]
    for qq in qs:
        qq.set_stream(torch.cuda.Stream())
        assert qq.summarize() == total
    W = 1000
    errs = []

    def work(k):
        try:
            for r0 in range(k * W, total, 2 * W):
                host = [torch.empty(W, dtype=c.dtype, pin_memory=True) for c in ref]
                got = qs[k].desummarize(r0, W, out=host)
                for a, b in zip(got, ref):
                    assert torch.equal(a, b[r0:r0 + a.shape[0]])
        except Exception as e:   # reported on the main thread
            errs.append(e)
    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for qq in qs:
        qq.close()
    run.close()


def test_emit_autotuner_picks_a_choice_and_results_stay_exact(kctx, tmp_path):
    """tune_emit times the emit's rows per thread on a real window, caches
    the choice per GPU and result shape, and leaves it set; the rows are the
    oracle's whichever it picks."""
    from paper_2206_10435_gb300 import autotune, gj
    q = G.chain3_uniform(seed=31, rows=3000, end_domain=600, mid_domain=50)
    run = Run(kctx, q)
    run.summarize()
    cache = str(tmp_path / "tune.json")
    first = autotune.tune_emit(kctx, run.q, window=1 << 16, reps=1, cache_path=cache)
    assert first["rpt"] in (2, 4, 8) and not first["cached"]
    assert set(first["candidates_ms"]) == {"2", "4", "8"}
    again = autotune.tune_emit(kctx, run.q, window=1 << 16, reps=1, cache_path=cache)
    assert again["cached"] and again["rpt"] == first["rpt"]
    ref = O.join(q)
    cols, rids = run.rows()
    assert np.array_equal(rids, ref.rowids)
    for a, b in zip(cols, O.columns(q, ref.rowids)):
        assert np.array_equal(a, b)
    kctx.set_option(gj.GJ_OPT_EMIT_ROWS_PER_THREAD, 4)
    run.close()
