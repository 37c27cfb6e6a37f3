"""The seeded input generators (paper_2206_10435_gb300/datagen.py) against
the input recipe they stand for: the same seed gives the same tables (the
oracle and the GPU path see identical inputs), keys stay in their domains,
Zipf ranks follow P(r) ~ (r+1)^-s, the star's dimensions hold Poisson copies
of every key, and the duplicated form repeats every row."""
import numpy as np
import pytest

from paper_2206_10435_gb300 import datagen as G


def _same(q1, q2):
    assert [R.attrs for R in q1.relations] == [R.attrs for R in q2.relations]
    for R1, R2 in zip(q1.relations, q2.relations):
        for a, b in zip(R1.keys + R1.payloads, R2.keys + R2.payloads):
            assert a.dtype == b.dtype and np.array_equal(a, b)


@pytest.mark.parametrize("make", [
    lambda seed: G.chain5_zipf(seed=seed, rows=5000, domain=3000),
    lambda seed: G.chain3_uniform(seed=seed, rows=2000),
    lambda seed: G.triangle_query(seed, [800, 900, 700], domain=50, s=0.6),
    lambda seed: G.star_poisson(seed=seed, fact_rows=4000, domain=500),
    lambda seed: G.random_tree_query(seed, 4, max_rows=6, domain=3),
])
def test_same_seed_same_tables_other_seed_other_tables(make):
    _same(make(11), make(11))
    a, b = make(11), make(12)
    assert any(not np.array_equal(x, y) for R1, R2 in zip(a.relations, b.relations)
               for x, y in zip(R1.keys, R2.keys))


def test_chain_keys_stay_in_their_domains_and_payloads_have_their_width():
    q = G.chain5_zipf(seed=3, rows=20000, domain=1000)
    assert len(q.relations) == 5
    for i, R in enumerate(q.relations):
        assert R.attrs == [i, i + 1]
        for k in R.keys:
            assert k.dtype == np.int32 and k.min() >= 0 and k.max() < 1000
        assert [p.dtype for p in R.payloads] == [np.int64]
    q3 = G.chain3_uniform(seed=3, rows=4000, end_domain=700, mid_domain=90)
    assert [int(R.keys[0].max()) < d0 and int(R.keys[1].max()) < d1
            for R, (d0, d1) in zip(q3.relations, [(700, 90), (90, 90), (90, 700)])] == [True] * 3
    assert [p.dtype for R in q3.relations for p in R.payloads] == [np.int32] * 3


@pytest.mark.parametrize("s", [0.7, 1.1, 1.5])
def test_zipf_ranks_follow_the_power_law(s):
    # P(r) / P(r') = ((r'+1)/(r+1))^s: compare the frequencies of ranks 0..3
    rng = np.random.default_rng(5)
    n, D = 2_000_000, 1000
    r = G.zipf_ranks(rng, n, s, D)
    assert r.min() >= 0 and r.max() < D
    c = np.bincount(r, minlength=D).astype(np.float64)
    for a, b in [(0, 1), (0, 3), (1, 3)]:
        want = ((b + 1) / (a + 1)) ** s
        assert abs(c[a] / c[b] / want - 1) < 0.03, (a, b, c[a] / c[b], want)
    # the normalised law: P(0) = 1 / sum_r (r+1)^-s
    p0 = 1.0 / np.sum(np.arange(1, D + 1, dtype=np.float64) ** -s)
    assert abs(c[0] / n / p0 - 1) < 0.02


def test_zipf_keys_are_a_permutation_of_ranks_per_column():
    # heavy hitters of different columns land on different keys, but each
    # column's key frequencies are the rank frequencies relabelled
    rng = np.random.default_rng(9)
    k1 = G.zipf_keys(rng, 200_000, 1.1, 500)
    k2 = G.zipf_keys(rng, 200_000, 1.1, 500)
    f1 = np.sort(np.bincount(k1, minlength=500))[::-1]
    f2 = np.sort(np.bincount(k2, minlength=500))[::-1]
    assert np.argmax(np.bincount(k1)) != np.argmax(np.bincount(k2))   # seeded: 147 vs 210
    assert abs(f1[0] / f2[0] - 1) < 0.05
    r = G.zipf_ranks(np.random.default_rng(10), 200_000, 1.1, 500)
    fr = np.sort(np.bincount(r, minlength=500))[::-1]
    assert np.abs(f1[:20] / fr[:20] - 1).max() < 0.1
    aligned = G.zipf_keys(np.random.default_rng(9), 200_000, 1.1, 500, aligned=True)
    assert np.argmax(np.bincount(aligned)) == 0


def test_star_dimensions_hold_poisson_copies_of_every_key():
    lam, D = 2.0, 20000
    q = G.star_poisson(seed=4, fact_rows=50000, domain=D, n_dims=4, lam=lam)
    F, dims = q.relations[0], q.relations[1:]
    assert F.attrs == [1, 2, 3, 4] and all(d.attrs == [j + 1] for j, d in enumerate(dims))
    for k in F.keys:
        assert k.min() >= 0 and k.max() < D
    for d in dims:
        copies = np.bincount(d.keys[0], minlength=D)
        assert copies.shape[0] == D
        assert abs(copies.mean() / lam - 1) < 0.03           # Poisson mean
        assert abs(copies.var() / lam - 1) < 0.06            # and variance
        assert abs((copies == 0).mean() / np.exp(-lam) - 1) < 0.08
        assert not np.all(np.diff(d.keys[0]) >= 0)          # shuffled


def test_duplicated_form_repeats_every_row():
    base = G.chain_sensitivity(rows=3000, domain=400, hops=3)
    dup = G.duplicate_rows(base, times=3)
    for R, Rd in zip(base.relations, dup.relations):
        assert Rd.n_rows == 3 * R.n_rows
        for a, b in zip(R.keys + R.payloads, Rd.keys + Rd.payloads):
            assert np.array_equal(b, np.tile(a, 3))
