"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts, offsets, multiplicities, summary levels and materialised rows are
integers and must match bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests import golden_fig
from tests.gpu_util import Run, check_canonical_window, device_columns, to_u64

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


def full_parity(ctx, q, check_levels=True, windows=()):
    """Everything the oracle can materialise, compared exactly."""
    run = Run(ctx, q)
    c = O.count(q, rows=True)
    total = run.summarize()
    assert total == c.total
    if total:
        j = O.join(q)
        ref_cols = O.columns(q, j.rowids)
        cols, rids = run.rows()
        assert np.array_equal(rids, j.rowids)
        for a, b in zip(cols, ref_cols):
            assert np.array_equal(a, b)
        # arbitrary windows, including ragged tails and single rows
        for (r0, n) in windows:
            if r0 >= total:
                continue
            cw, rw = run.rows(r0, n)
            m = min(n, total - r0)
            assert np.array_equal(rw, j.rowids[r0:r0 + m])
            for a, b in zip(cw, ref_cols):
                assert np.array_equal(a, b[r0:r0 + m])
        if check_levels:
            lv = O.gfjs_levels(q, j.rowids)
            for l in range(len(lv)):
                val, freq, off = run.q.level(l, 0, total)
                assert np.array_equal(val.cpu().numpy(), lv[l].value)
                assert np.array_equal(to_u64(freq), lv[l].freq)
                assert np.array_equal(to_u64(off), lv[l].offset)
    # per key-tuple multiplicities
    gm = O.group_mult_from_counts(q, c)
    for rel in range(len(q.relations)):
        tab = run.group_table(rel)
        keys, mult = gm[rel]
        assert len(tab) == keys.shape[0]
        for k, m in zip(keys.tolist(), mult.tolist()):
            assert tab[tuple(k)][1] == int(m), (rel, k)
    run.close()
    return total


def test_figure1_on_gpu(ctx):
    q, result, gfjs, _ = golden_fig.load()
    run = Run(ctx, q)
    assert run.summarize() == 32
    cols, rids = run.rows()
    assert list(zip(*[c.tolist() for c in cols])) == result
    for l, name in enumerate("ABCD"):
        val, freq, off = run.q.level(l, 0, 32)
        assert list(zip(val.tolist(), to_u64(freq).tolist())) == gfjs[name]
    t1 = run.group_table(0)
    assert t1[(3, 3)] == (8, 8) and t1[(3, 4)] == (24, 24) and t1[(0, 0)] == (0, 0)
    t2 = run.group_table(1)
    assert t2[(4, 3)][1] == 16
    run.close()


def tiny_queries():
    qs = []
    for seed in range(160):
        n_rel = 1 + seed % 5
        qs.append(G.random_tree_query(seed, n_rel, max_rows=5 if n_rel <= 3 else 4,
                                      domain=3 if n_rel <= 2 else 2, max_new=2,
                                      min_rows=0 if seed % 7 == 0 else 1))
    return qs


@pytest.mark.parametrize("q", tiny_queries(), ids=lambda q: q.name)
def test_tiny_random_trees(ctx, q):
    full_parity(ctx, q, windows=[(0, 1), (1, 2), (3, 5)])


@pytest.mark.parametrize("seed", range(12))
def test_small_random_trees_several_tiles(ctx, seed):
    # a few thousand result rows: several emit/expand tiles and ragged tails
    q = G.random_tree_query(1000 + seed, 2 + seed % 4, max_rows=60, domain=6, max_new=2,
                            min_rows=20)
    full_parity(ctx, q, windows=[(0, 1000), (999, 1025), (2047, 3001)])


def test_chain3_uniform_full(ctx):
    q = G.chain3_uniform()
    total = full_parity(ctx, q, windows=[(0, 1 << 18), (1 << 18, 1 << 18), (777_777, 1 << 20)])
    assert total == O.count(q).total


@pytest.mark.parametrize("s", [0.0, 1.1, 1.5])
def test_chain5_zipf_reduced(ctx, s):
    q = G.chain5_zipf(rows=20_000, domain=20_000, s=s)
    full_parity(ctx, q, check_levels=True, windows=[(12345, 100_000)])


def test_star_reduced(ctx):
    q = G.star_poisson(fact_rows=30_000, domain=10_000)
    full_parity(ctx, q, windows=[(5, 4097)])


def test_empty_relation(ctx):
    q = G.chain3_uniform(rows=100, end_domain=10, mid_domain=5)
    q.relations[1] = G.Relation("R2", [1, 2], [np.zeros(0, np.int32)] * 2, [np.zeros(0, np.int32)])
    run = Run(ctx, q)
    assert run.summarize() == 0
    cols, rids = run.rows(0, 10)
    assert all(c.shape[0] == 0 for c in cols)
    run.close()


def _all_equal_star(sizes, value=7):
    rels = [G.Relation(f"R{i}", [0], [np.full(n, value, np.int32)]) for i, n in enumerate(sizes)]
    return G.Query("allequal", rels)


def test_largest_exact_count(ctx):
    run = Run(ctx, _all_equal_star([2, 7, 7, 73, 127, 337, 92737, 649657]))
    assert run.summarize() == (1 << 64) - 2
    run.close()


def test_overflow_reported(ctx):
    from paper_2206_10435_gb300 import gj
    for sizes in ([3, 5, 17, 257, 641, 65537, 6700417], [256] * 9):
        run = Run(ctx, _all_equal_star(sizes))
        with pytest.raises(gj.GJError) as e:
            run.summarize()
        assert e.value.status == gj.GJ_ERR_OVERFLOW
        run.close()
    q = G.chain5_zipf(rows=10**6, domain=10**5, aligned=True)
    run = Run(ctx, q)
    with pytest.raises(gj.GJError) as e:
        run.summarize()
    assert e.value.status == gj.GJ_ERR_OVERFLOW
    run.close()


def test_dead_branch_does_not_overflow(ctx):
    rels = [G.Relation("R0", [0], [np.array([1, 1, 1], np.int32)])]
    rels.append(G.Relation("R1", [0, 1], [np.full(256, 2, np.int32), np.zeros(256, np.int32)]))
    for i in range(2, 9):
        rels.append(G.Relation(f"R{i}", [1], [np.zeros(256, np.int32)]))
    rels.append(G.Relation("R9", [0], [np.array([1, 2], np.int32)]))
    run = Run(ctx, G.Query("dead", rels))
    assert run.summarize() == 0
    run.close()


def test_rejects_disconnected_and_projected_cycles(ctx):
    # a relation sharing nothing is a cross product; a cyclic query cannot
    # project attributes away early (only a join tree can); the 4-cycle
    # itself is answered (tests/test_gpu_cyclic.py)
    from paper_2206_10435_gb300 import gj
    a = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    r = ctx.load_relation([a, a], [0, 1])
    s = ctx.load_relation([a, a], [1, 2])
    t = ctx.load_relation([a, a], [2, 3])
    v = ctx.load_relation([a, a], [3, 0])
    u = ctx.load_relation([a], [9])
    ctx.query([r, s, t, v]).close()
    with pytest.raises(gj.GJError) as e:
        ctx.query([r, s, t, v], drop_attrs=[3])
    assert e.value.status in (gj.GJ_ERR_INVALID, gj.GJ_ERR_NOT_ACYCLIC)
    with pytest.raises(gj.GJError) as e:
        ctx.query([r, u])
    assert e.value.status == gj.GJ_ERR_INVALID
    for x in (r, s, t, v, u):
        ctx.release_relation(x)


def test_factor_matches_stable_sort(ctx):
    rng = np.random.default_rng(3)
    n = 300_000
    cols = [rng.integers(-5, 1 << 20, n, dtype=np.int32), rng.integers(-(1 << 31), (1 << 31) - 1, n,
                                                                          dtype=np.int32),
            rng.integers(0, 3, n, dtype=np.int32)]
    dev = [torch.from_numpy(c).cuda() for c in cols]
    rid = ctx.load_relation(dev, [0, 1, 2])
    for order in ([0, 1, 2], [2, 0, 1], [1, 2, 0]):
        perm, gstart, gkey = ctx.factor_export(rid, n, 3, order)
        ref = np.lexsort([cols[c] for c in reversed(order)])   # stable
        assert np.array_equal(perm.cpu().numpy(), ref)
        srt = np.stack([cols[c][ref] for c in range(3)], axis=1)
        head = np.ones(n, bool)
        head[1:] = (srt[1:] != srt[:-1]).any(axis=1)
        starts = np.flatnonzero(head)
        assert np.array_equal(gstart.cpu().numpy()[:-1], starts)
        assert int(gstart[-1]) == n
        assert np.array_equal(gkey.cpu().numpy().T, srt[starts])
    ctx.release_relation(rid)


def _check_factor(ctx, rid, cols, order, n):
    perm, gstart, gkey = ctx.factor_export(rid, n, len(cols), order)
    ref = np.lexsort([cols[c] for c in reversed(order)])   # stable: row id breaks ties
    assert np.array_equal(perm.cpu().numpy(), ref)
    srt = np.stack([cols[c][ref] for c in range(len(cols))], axis=1)
    head = np.ones(n, bool)
    head[1:] = (srt[1:] != srt[:-1]).any(axis=1)
    starts = np.flatnonzero(head)
    assert np.array_equal(gstart.cpu().numpy()[:-1], starts)
    assert int(gstart[-1]) == n
    assert np.array_equal(gkey.cpu().numpy().T, srt[starts])


@pytest.mark.parametrize("long_run", [False, True])
def test_factor_wide_keys_match_stable_sort(ctx, long_run):
    """Keys of three 22-bit columns (66 bits: with the row id they need two
    words).  The rows are sorted by the leading columns, then run by run by
    the rest; runs of up to 256 rows are sorted by one warp.  A run longer
    than that (long_run) sends the factor down the two-word path instead;
    both give the stable sort."""
    rng = np.random.default_rng(11)
    n = 100_000
    spread = lambda k: rng.choice(np.linspace(-(1 << 21), (1 << 21) - 1, k).astype(np.int32), n)
    c0, c1 = spread(40), spread(40)
    c2 = rng.integers(-(1 << 21), 1 << 21, n, dtype=np.int32)
    c2[::7] = 5                       # repeated full keys: rows tie on the key
    if long_run:
        c0[:1000] = c0[0]
        c1[:1000] = c1[0]
    cols = [c0, c1, c2]
    rid = ctx.load_relation([torch.from_numpy(c).cuda() for c in cols], [0, 1, 2])
    for order in ([0, 1, 2], [2, 0, 1], [1, 0, 2]):
        _check_factor(ctx, rid, cols, order, n)
    ctx.release_relation(rid)


def _all_group_mult(q, c, run, rel):
    """Every group of relation rel against the oracle's counting pass, in
    O(rows): every row of a group holds the group's key tuple, groups are
    strictly increasing in the factor's column order (so they are the
    distinct key tuples), and a group's multiplicity is the sum of the
    oracle's per-row multiplicities over its rows.  Returns (keys in
    declared column order, multiplicities) in group order."""
    R = q.relations[rel]
    order = run.factor_order(rel)
    perm, gstart, gkey = run.ctx.factor_export(run.ids[rel], R.n_rows, len(R.keys), order)
    _, m, _ = run.q.summary_groups(rel)
    perm = perm.cpu().numpy().astype(np.int64)
    gs = gstart.cpu().numpy().astype(np.int64)
    keys = gkey.cpu().numpy()                     # [column][group]
    G = keys.shape[1]
    sizes = np.diff(gs)
    assert sizes.min() >= 1 and gs[-1] == R.n_rows
    for col in range(len(R.keys)):
        assert np.array_equal(R.keys[col][perm], np.repeat(keys[col], sizes)), (rel, col)
    if G > 1:   # strictly increasing, most significant column first
        diff = np.zeros(G - 1, dtype=np.int8)
        for col in reversed(order):
            d = np.sign(keys[col][1:].astype(np.int64) - keys[col][:-1])
            diff = np.where(d != 0, d, diff)
        assert (diff > 0).all(), rel
    row_mult = c.mult[rel].astype(np.uint64)[perm]
    want = np.add.reduceat(row_mult, gs[:-1]) if G else np.zeros(0, np.uint64)
    got = to_u64(m)
    assert np.array_equal(got, want), rel
    return keys.T, got


def test_chain5_zipf_full_size(ctx):
    """5-chain, 10^7 rows per table, Zipf(1.1) over 10^6: exact total, the
    multiplicity of every group of every relation against the oracle's
    counting pass, GFJS level 0 against the per-value marginal of K0, and
    every 2^28-row window checked by properties that pin it to the sorted
    result."""
    q = G.chain5_zipf()
    c = O.count(q, rows=True)
    run = Run(ctx, q)
    total = run.summarize()
    assert total == c.total
    got = [_all_group_mult(q, c, run, rel) for rel in range(5)]
    # level 0 (V[0] = K0, held by R1's first column): one run per K0 value,
    # its frequency the marginal of that value = summed multiplicities of
    # R1's key tuples with it (Section 1.2)
    allk, m = got[0]
    pl = O.plan(q)
    col = q.relations[0].attrs.index(pl.V[0])
    vals, inv = np.unique(allk[:, col], return_inverse=True)
    marg = np.zeros(vals.shape[0], dtype=np.uint64)
    np.add.at(marg, inv.reshape(-1), m)
    live = marg > 0
    # runs are returned by the window of result rows they start in; the
    # windows partition the level
    parts = [run.q.level(0, r0, 1 << 28, cap=int(live.sum())) for r0 in range(0, total, 1 << 28)]
    val = np.concatenate([p[0].cpu().numpy() for p in parts])
    freq = np.concatenate([to_u64(p[1]) for p in parts])
    off = np.concatenate([to_u64(p[2]) for p in parts])
    assert np.array_equal(val, vals[live].astype(np.int32))
    assert np.array_equal(freq, marg[live])
    want_off = np.concatenate([[0], np.cumsum(marg[live])[:-1]]).astype(np.uint64)
    assert np.array_equal(off, want_off)
    dev = device_columns(torch, q)
    W = 1 << 28
    last = None
    done = 0
    for r0 in range(0, total, W):
        out, rids = run.q.desummarize(r0, W, rowids=True)
        last = check_canonical_window(torch, q, pl, dev, out, rids, last)
        assert out[0].shape[0] == min(W, total - r0)
        done += out[0].shape[0]
        del out, rids
    assert done == total
    run.close()


def test_star_full_size(ctx):
    """Star, fact table 10^8 rows: exact total, the multiplicity of every
    group of the fact and dimension tables against the oracle's counting
    pass, and every window checked by the canonical-order properties."""
    q = G.star_poisson()
    c = O.count(q, rows=True)
    run = Run(ctx, q)
    total = run.summarize()
    assert total == c.total
    for rel in range(len(q.relations)):
        _all_group_mult(q, c, run, rel)
    dev = device_columns(torch, q)
    pl = O.plan(q)
    W = 1 << 28
    last = None
    done = 0
    for r0 in range(0, total, W):
        out, rids = run.q.desummarize(r0, W, rowids=True)
        last = check_canonical_window(torch, q, pl, dev, out, rids, last)
        done += out[0].shape[0]
        del out, rids
    assert done == total
    run.close()


def shape_queries():
    qs = []
    for seed in range(40):
        n_rel = 2 + seed % 4
        qs.append(G.random_tree_query(500 + seed, n_rel, max_rows=5 if n_rel <= 3 else 4,
                                      domain=3, max_new=2, min_rows=1, max_shared=3,
                                      spread=(seed % 3) * 600_000_007 % 2_000_000_000 // 3))
    return qs


@pytest.mark.parametrize("q", shape_queries(), ids=lambda q: q.name)
def test_multi_attribute_separators_and_wide_ranges(ctx, q):
    # separators of 2-3 attributes (binary-search links) and keys spread over
    # the int32 range (no dense link table)
    full_parity(ctx, q, windows=[(0, 1), (2, 3)])


@pytest.mark.parametrize("seed", [0, 1, 3, 4, 5, 6])
def test_many_relations(ctx, seed):
    # 9-12 relations: beyond the templated emit kernels (generic path)
    q = G.random_tree_query(900 + seed, 9 + seed % 4, max_rows=5, domain=2, max_new=1,
                            min_rows=4)
    assert O.count(q).total > 0
    full_parity(ctx, q, windows=[(0, 7), (5, 1000)])


@pytest.mark.parametrize("seed", range(4))
def test_larger_random_trees_with_multi_attribute_separators(ctx, seed):
    q = G.random_tree_query(1300 + seed, 3 + seed % 3, max_rows=80, domain=5, max_new=2,
                            min_rows=30, max_shared=2, spread=seed * 1_000_003)
    full_parity(ctx, q, windows=[(0, 1000), (1001, 1025)])


@pytest.mark.parametrize("seed", range(6))
def test_keys_at_the_int32_ends(ctx, seed):
    # every key value at INT32_MIN, INT32_MIN + 1, -1, 0, INT32_MAX - 1 or
    # INT32_MAX: key ranges span 2^32 - 1, sort words and links must not wrap,
    # and the result follows the signed order
    base = G.random_tree_query(2300 + seed, 2 + seed % 4, max_rows=60, domain=5, max_new=2,
                               min_rows=20, max_shared=1 + seed % 2)
    q = G.extreme_keys(base, seed)
    assert O.count(q).total == O.count(base).total
    full_parity(ctx, q, windows=[(0, 1), (3, 700)])


def test_window_contract(ctx):
    """Windows of gj_desummarize and gj_level: GJ_ERR_STATE before the
    summary; empty windows and windows at or past |Q| write nothing; a
    window reaching past |Q| is clipped (n_rows up to 2^64 - 1); a level
    index out of range is invalid; too small a capacity reports
    GJ_ERR_CAPACITY; a clipped window of 2^31 rows or more is invalid."""
    from paper_2206_10435_gb300 import gj
    q = G.chain3_uniform(seed=5, rows=300, end_domain=30, mid_domain=6)
    run = Run(ctx, q)
    for call in (lambda: run.q.desummarize(0, 4), lambda: run.q.level(0, 0, 4, cap=4)):
        with pytest.raises(gj.GJError) as e:
            call()
        assert e.value.status == gj.GJ_ERR_STATE
    total = run.summarize()
    assert total == O.count(q).total > 3
    j = O.join(q)
    ref = O.columns(q, j.rowids)
    for r0, n in [(0, 0), (total, 5), (total + 1000, 5), (1 << 63, 5)]:
        assert all(c.numel() == 0 for c in run.q.desummarize(r0, n))
        assert run.q.level(0, r0, n, cap=4)[0].numel() == 0
    cols = run.q.desummarize(total - 3, (1 << 64) - 1, out=run.q.alloc_columns(3))
    assert cols[0].shape[0] == 3
    for a, b in zip(cols, ref):
        assert np.array_equal(a.cpu().numpy(), b[total - 3:])
    lv = O.gfjs_levels(q, j.rowids)
    with pytest.raises(gj.GJError) as e:
        run.q.level(len(lv), 0, total)
    assert e.value.status == gj.GJ_ERR_INVALID
    k = lv[0].value.shape[0]
    assert k > 1
    with pytest.raises(gj.GJError) as e:
        run.q.level(0, 0, total, cap=k - 1)
    assert e.value.status == gj.GJ_ERR_CAPACITY
    assert np.array_equal(run.q.level(0, 0, total, cap=k)[0].cpu().numpy(), lv[0].value)
    run.close()
    # all keys equal: |Q| = 2000^3 > 2^31, so a window of 2^31 rows is refused
    # before anything is written
    big = G.Query("equal3", [G.Relation(f"R{i}", [i, i + 1], [np.full(2000, 7, np.int32)] * 2, [])
                             for i in range(3)], {a: f"X{a}" for a in range(4)})
    run = Run(ctx, big)
    assert run.summarize() == 2000 ** 3 == O.count(big).total
    for call in (lambda: run.q.desummarize(5, 1 << 31, out=run.q.alloc_columns(1)),
                 lambda: run.q.level(2, 0, 1 << 31, cap=1)):
        with pytest.raises(gj.GJError) as e:
            call()
        assert e.value.status == gj.GJ_ERR_INVALID
    # rows past 2^32 (64-bit digit arithmetic): all keys equal, so row r is
    # the row-id tuple (r // 2000^2, r // 2000 % 2000, r % 2000)
    r0 = (1 << 32) + 5
    cols, rids = run.q.desummarize(r0, 2, out=run.q.alloc_columns(2), rowids=True)
    assert [c.cpu().tolist() for c in cols] == [[7, 7]] * 4
    for i, r in enumerate((r0, r0 + 1)):
        assert [int(t[i]) for t in rids] == [r // 2000 ** 2, r // 2000 % 2000, r % 2000]
    run.close()


@pytest.mark.parametrize("hops", [3, 4])
def test_sensitivity_variants(ctx, hops):
    # Section 4.2: the duplicated form multiplies |Q| by 2^k; the extra hop
    # adds a join; both stay exact
    base = G.chain_sensitivity(rows=4000, domain=3000, hops=hops)
    dup = G.duplicate_rows(base)
    tb = full_parity(ctx, base, check_levels=False)
    td = full_parity(ctx, dup, check_levels=False)
    assert td == tb * 2 ** hops
