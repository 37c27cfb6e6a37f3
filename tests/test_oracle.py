"""Pins the CPU oracle to facts fixed outside itself: the paper's worked
example (Figures 1 and 2, Section 1.1), brute-force nested loops over every
row combination on tiny inputs, closed forms, and the 2^64 boundary."""
import itertools
from collections import Counter

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G
from tests import golden_fig

CAP = (1 << 64) - 1


# ------------------------------------------------------------------ helpers

def brute_force(q):
    """All row-id tuples whose rows agree on every shared attribute (the
    definition of the natural join, checked pairwise over ALL relations,
    not along a tree)."""
    rels = q.relations
    k = len(rels)
    pairs = []
    for i in range(k):
        for j in range(i + 1, k):
            for ci, a in enumerate(rels[i].attrs):
                if a in rels[j].attrs:
                    pairs.append((i, ci, j, rels[j].attrs.index(a)))
    out = []
    for combo in itertools.product(*[range(R.n_rows) for R in rels]):
        if all(rels[i].keys[ci][combo[i]] == rels[j].keys[cj][combo[j]]
               for i, ci, j, cj in pairs):
            out.append(combo)
    return out


def value_of(q, combo, attr):
    for j, R in enumerate(q.relations):
        if attr in R.attrs:
            return int(R.keys[R.attrs.index(attr)][combo[j]])
    raise KeyError(attr)


def canonical(q, tuples, V):
    return sorted(tuples, key=lambda t: tuple(value_of(q, t, a) for a in V) + tuple(t))


def levels_by_definition(q, tuples, V):
    """Per-prefix runs of the sorted result (Def. 1 / Algorithm 4)."""
    out = []
    for l in range(len(V)):
        runs = []
        prev = None
        for i, t in enumerate(tuples):
            pre = tuple(value_of(q, t, a) for a in V[:l + 1])
            if pre != prev:
                runs.append([pre[-1], 0, i])
                prev = pre
            runs[-1][1] += 1
        out.append(runs)
    return out


def tiny_queries():
    qs = []
    for seed in range(160):
        n_rel = 1 + seed % 5
        qs.append(G.random_tree_query(seed, n_rel, max_rows=5 if n_rel <= 3 else 4,
                                      domain=3 if n_rel <= 2 else 2, max_new=2,
                                      min_rows=0 if seed % 7 == 0 else 1))
    return qs


# ------------------------------------------------------------------ Figure 1 / 2

def test_figure1_plan_is_chain_rooted_at_A():
    q, *_ = golden_fig.load()
    pl = O.plan(q)
    assert pl.parent == [-1, 0, 1]
    assert pl.V == [0, 1, 2, 3]          # A, B, C, D (root A, Section 3.3 example)


def test_figure1_join_size_and_result():
    q, result, _, _ = golden_fig.load()
    c = O.count(q)
    assert c.total == 32 and not c.overflow
    j = O.join(q)
    cols = O.columns(q, j.rowids)
    got = list(zip(*[c_.tolist() for c_ in cols]))
    assert got == result                  # Figure 2, rows 0..31


def test_figure1_gfjs_levels():
    q, _, gfjs, _ = golden_fig.load()
    j = O.join(q)
    lv = O.gfjs_levels(q, j.rowids)
    for l, name in enumerate("ABCD"):
        assert list(zip(lv[l].value.tolist(), lv[l].freq.tolist())) == gfjs[name]
        assert int(lv[l].freq.sum()) == 32          # equal sums per column (Def. 1)
        off = np.concatenate([[0], np.cumsum(lv[l].freq)[:-1]])
        assert (lv[l].offset == off).all()


def test_figure1_unneeded_intermediate_tuples():
    q, _, _, facts = golden_fig.load()
    j = O.join(q)
    # the cascade joins T1 with T2 first; tuples of that intermediate result
    # that never reach the final result are the UIR of Section 1.1
    used = {(int(a), int(b)) for a, b in j.rowids[:, :2].tolist()}
    uir = j.intermediate[1] - len(used)
    expect = [int(f[3]) for f in facts if f[0] == "uir"][0]
    assert uir == expect == 15
    T1 = q.relations[0]
    assert int((T1.keys[0] == 3).sum()) == 6
    assert int((O.columns(q, j.rowids)[0] == 3).sum()) == 32


def test_figure1_generator_values():
    """Messages and root weights of the running example (Section 3.3):
    fac = 1 at the leaf, phi(C) from T3, phi(B) from T2 and T3, the root
    marginal p(A) = (a3, 32), and the multiplicity of (b4, c3) = 16."""
    q, *_ = golden_fig.load()
    c = O.count(q, rows=True)
    T2, T3 = q.relations[1], q.relations[2]
    assert (c.up[2] == 1).all()                               # leaf rows
    msg_c = Counter(int(x) for x in T3.keys[0])
    assert dict(msg_c) == {1: 4, 2: 4, 3: 2, 4: 2}
    msg_b = Counter()
    for r in range(T2.n_rows):
        msg_b[int(T2.keys[0][r])] += int(c.up[1][r])
    assert {b: v for b, v in msg_b.items() if v} == {2: 12, 3: 4, 4: 6}
    gm = O.group_mult_from_counts(q, c)
    t1 = {tuple(k): int(m) for k, m in zip(gm[0][0].tolist(), gm[0][1])}
    assert t1[(3, 3)] == 8 and t1[(3, 4)] == 24 and t1[(0, 0)] == 0
    t2 = {tuple(k): int(m) for k, m in zip(gm[1][0].tolist(), gm[1][1])}
    assert t2[(4, 3)] == 16 and t2[(4, 4)] == 8 and t2[(3, 2)] == 8


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("q", tiny_queries(), ids=lambda q: q.name)
def test_oracle_matches_nested_loops(q):
    pl = O.plan(q)
    bf = canonical(q, brute_force(q), pl.V)
    c = O.count(q, rows=True)
    assert c.total == len(bf) and not c.overflow
    if not bf:
        return
    j = O.join(q)
    assert [tuple(t) for t in j.rowids.tolist()] == [tuple(t) for t in bf]
    # materialised columns: V values, then payloads by row id
    cols = O.columns(q, j.rowids)
    for i, t in enumerate(bf[:50]):
        assert [int(cols[v][i]) for v in range(len(pl.V))] == [value_of(q, t, a) for a in pl.V]
        pc = len(pl.V)
        for jj, R in enumerate(q.relations):
            for p in R.payloads:
                assert int(cols[pc][i]) == int(p[t[jj]])
                pc += 1
    # summary levels
    lv = O.gfjs_levels(q, j.rowids)
    ref = levels_by_definition(q, bf, pl.V)
    for l in range(len(pl.V)):
        assert [list(x) for x in zip(lv[l].value.tolist(), lv[l].freq.tolist(),
                                     lv[l].offset.tolist())] == ref[l]
    # per key-tuple multiplicities, two ways
    gm_c = O.group_mult_from_counts(q, c)
    gm_r = O.group_mult_from_rows(q, j.rowids)
    for jj, R in enumerate(q.relations):
        cnt = Counter(tuple(int(R.keys[ci][t[jj]]) for ci in range(len(R.keys))) for t in bf)
        got = {tuple(k): int(m) for k, m in zip(gm_c[jj][0].tolist(), gm_c[jj][1])}
        assert {k: v for k, v in got.items() if v} == dict(cnt)
        assert (gm_c[jj][1] == gm_r[jj][1]).all()
        assert int(gm_c[jj][1].sum()) == c.total   # each relation sums to |Q|


def droppable(q):
    """Attributes held by exactly one relation, keeping at least one key
    column on the root (the attributes early projection may delete)."""
    rels = q.relations
    one = [a for R in rels for a in R.attrs if sum(S.attrs.count(a) for S in rels) == 1]
    if rels and all(a in one for a in rels[0].attrs):
        one = [a for a in one if a != rels[0].attrs[0]]
    return sorted(set(one))


@pytest.mark.parametrize("q", [q for q in tiny_queries() if droppable(q)][:80],
                         ids=lambda q: q.name)
def test_early_projection_matches_nested_loops(q):
    """Section 3.7: deleting attributes held by one relation keeps the bag of
    row-id tuples; rows are ordered by the remaining variables, then row ids;
    levels are the per-prefix runs over the remaining variables."""
    cand = droppable(q)
    for drop in (cand[:1], cand):
        full = O.plan(q)
        pl = O.plan(q, drop)
        assert pl.V == [a for a in full.V if a not in drop]
        bf = canonical(q, brute_force(q), pl.V)
        if not bf:
            continue
        j = O.join(q, drop=drop)
        assert [tuple(t) for t in j.rowids.tolist()] == [tuple(t) for t in bf]
        jf = O.join(q)
        assert sorted(map(tuple, jf.rowids.tolist())) == sorted(map(tuple, j.rowids.tolist()))
        cols = O.columns(q, j.rowids, drop)
        assert len(cols) == len(pl.V) + sum(len(R.payloads) for R in q.relations)
        for i, t in enumerate(bf[:50]):
            assert [int(cols[v][i]) for v in range(len(pl.V))] == [value_of(q, t, a) for a in pl.V]
        lv = O.gfjs_levels(q, j.rowids, drop)
        ref = levels_by_definition(q, bf, pl.V)
        for l in range(len(pl.V)):
            assert [list(x) for x in zip(lv[l].value.tolist(), lv[l].freq.tolist(),
                                         lv[l].offset.tolist())] == ref[l]


def test_early_projection_rejects_shared_attributes():
    q, _, _, _ = golden_fig.load()
    with pytest.raises(ValueError):
        O.plan(q, drop=[q.relations[0].attrs[1]])   # B joins R1 and R2
    pl = O.plan(q, drop=[q.relations[0].attrs[0], q.relations[-1].attrs[-1]])
    assert len(pl.V) == len(O.plan(q).V) - 2


def tiny_triangles():
    qs = []
    for seed in range(60):
        q = G.triangle_query(7000 + seed, [1 + seed % 5, 1 + (seed // 5) % 4, 1 + (seed // 3) % 5],
                             domain=2 + seed % 3, payload_dtype=np.int32 if seed % 2 else np.int64)
        if seed % 4 in (1, 3):   # columns in another declared order
            r = 2 if seed % 4 == 1 else 0
            R = q.relations[r]
            q.relations[r] = G.Relation(R.name, R.attrs[::-1], R.keys[::-1], R.payloads)
        qs.append(q)
    return qs


@pytest.mark.parametrize("q", tiny_triangles(), ids=lambda q: f"tri{id(q) % 997}")
def test_cyclic_triangle_matches_nested_loops(q):
    """The 3-cycle's result: every row combination agreeing on A, B and C,
    ordered by R0's columns, then C, then the row ids."""
    pl = O.plan(q)
    assert pl.cyclic and pl.V == list(q.relations[0].attrs) + [2]   # V = R0's columns, then C
    bf = canonical(q, brute_force(q), pl.V)
    assert O.count(q).total == len(bf)
    j = O.join(q)
    assert [tuple(t) for t in j.rowids.tolist()] == [tuple(t) for t in bf]
    cols = O.columns(q, j.rowids)
    for i, t in enumerate(bf[:50]):
        assert [int(cols[v][i]) for v in range(3)] == [value_of(q, t, a) for a in pl.V]
    lv = O.gfjs_levels(q, j.rowids)
    ref = levels_by_definition(q, bf, pl.V)
    for l in range(3):
        assert [list(x) for x in zip(lv[l].value.tolist(), lv[l].freq.tolist(),
                                     lv[l].offset.tolist())] == ref[l]


def _paper_triangle():
    """Section 3.2.1's example: T1(A,B), T2(B,C), T3(C,A) with the entries
    (a1,b1) x5, (b1,c1) x10, (c1,a1) x20, plus rows that close no cycle."""
    def rel(name, attrs, pairs):
        x = np.array([p[0] for p in pairs], np.int32)
        y = np.array([p[1] for p in pairs], np.int32)
        return G.Relation(name, attrs, [x, y], [np.arange(len(pairs), dtype=np.int64)])
    t1 = rel("T1", [0, 1], [(1, 1)] * 5 + [(2, 1), (1, 3)])
    t2 = rel("T2", [1, 2], [(1, 1)] * 10 + [(3, 7)])
    t3 = rel("T3", [2, 0], [(1, 1)] * 20 + [(1, 2), (7, 9)])
    return G.Query("paper_triangle", [t1, t2, t3], {0: "A", 1: "B", 2: "C"})


def test_cyclic_triangle_paper_example_gives_1000():
    # the joint potential's entry (a1, b1, c1) has frequency 5 * 10 * 20; the
    # added rows give one more entry (a2, b1, c1) of frequency 1 * 10 * 1, and
    # (a1, b3, c7) does not close (T3 holds (c7, a9), not (c7, a1))
    q = _paper_triangle()
    assert O.count(q).total == 5 * 10 * 20 + 1 * 10 * 1
    bf = canonical(q, brute_force(q), O.plan(q).V)
    assert len(bf) == 1010


def test_cyclic_triangle_all_equal_keys_gives_product():
    q = G.triangle_query(1, [7, 5, 3], domain=1)
    assert O.count(q).total == 7 * 5 * 3


@pytest.mark.parametrize("k,seed,s", [(2, 0, 0.0), (3, 1, 0.8), (4, 2, 1.3), (5, 3, 1.1), (5, 4, 0.0)])
def test_chain_counts_are_products_of_the_count_matrices(k, seed, s):
    # For R_i(K_{i-1}, K_i), i = 1..k, with M_i the pair-count matrix of R_i:
    # |Q| = 1' M_1 ... M_k 1, and a row (x, y) of R_i is in
    # (1' M_1 ... M_{i-1})[x] * (M_{i+1} ... M_k 1)[y] result tuples: the
    # upward and downward messages of the counting pass, by library matrix
    # products (Eq. 6-10's sum-product on a chain), independent of the oracle
    d = [7 + (seed + j) % 5 for j in range(k + 1)]
    q = G.chain_query(f"chain{k}", [40 + 17 * i for i in range(k)], d, [s] * (k + 1), None, 9300 + seed)
    M = []
    for i, R in enumerate(q.relations):
        m = np.zeros((d[i], d[i + 1]), np.int64)
        np.add.at(m, (R.keys[0].astype(np.int64), R.keys[1].astype(np.int64)), 1)
        M.append(m)
    left = [np.ones(d[0], np.int64)]
    for i in range(k):
        left.append(left[-1] @ M[i])
    right = [np.ones(d[k], np.int64)]
    for i in reversed(range(k)):
        right.insert(0, M[i] @ right[0])
    c = O.count(q, rows=True)
    assert c.total == int(left[k].sum()) == int(right[0].sum())
    for i, R in enumerate(q.relations):
        want = left[i][R.keys[0]] * right[i + 1][R.keys[1]]
        assert np.array_equal(c.mult[i].astype(np.int64), want), i


@pytest.mark.parametrize("seed,s", [(0, 0.0), (1, 0.9), (2, 1.5), (3, 0.4)])
def test_cyclic_triangle_size_is_the_trace_of_the_count_matrices(seed, s):
    # |R(A,B) join S(B,C) join T(C,A)| = sum over (a,b,c) of
    # n_R(a,b) n_S(b,c) n_T(c,a) = trace(M_R M_S M_T), with M the tables'
    # pair-count matrices: a library matrix product, independent of the
    # oracle's hash joins
    d = 12 + seed
    q = G.triangle_query(9100 + seed, [300, 250, 400], domain=d, s=s)
    M = []
    for R in q.relations:
        m = np.zeros((d, d), np.int64)
        np.add.at(m, (R.keys[0].astype(np.int64), R.keys[1].astype(np.int64)), 1)
        M.append(m)
    # R is (A,B), S is (B,C), T is (C,A)
    assert O.count(q).total == int(np.trace(M[0] @ M[1] @ M[2]))


def test_cyclic_triangle_complete_tripartite_closed_form():
    # every pair present m times in each table: |Q| = |A| |B| |C| m_R m_S m_T
    na, nb, nc, mr, ms, mt = 3, 4, 2, 2, 3, 1
    def full(xs, ys, m, attrs, name):
        x = np.repeat(np.array([u for u in xs for _ in ys], np.int32), m)
        y = np.repeat(np.array([v for _ in xs for v in ys], np.int32), m)
        return G.Relation(name, attrs, [x, y])
    A, B, C = range(-1, na - 1), range(10, 10 + nb), range(5, 5 + nc)
    q = G.Query("k_abc", [full(A, B, mr, [0, 1], "R"), full(B, C, ms, [1, 2], "S"),
                          full(C, A, mt, [2, 0], "T")], {0: "A", 1: "B", 2: "C"})
    assert O.count(q).total == na * nb * nc * mr * ms * mt
    j = O.join(q)
    assert j.rowids.shape[0] == na * nb * nc * mr * ms * mt


def tiny_cyclic():
    qs = []
    shapes = list(G.CYCLIC_SHAPES)
    for seed in range(70):
        shape = shapes[seed % len(shapes)]
        k = len(G.CYCLIC_SHAPES[shape])
        rows = [1 + (seed + 2 * i) % (4 if k <= 5 else 3) for i in range(k)]
        q = G.cyclic_query(7500 + seed, shape, rows, domain=2 + (seed // 7) % 2,
                           payload_dtype=np.int32 if seed % 2 else np.int64)
        if seed % 3 == 1:   # a relation's columns in another declared order
            r = seed % k
            R = q.relations[r]
            q.relations[r] = G.Relation(R.name, R.attrs[::-1], R.keys[::-1], R.payloads)
        qs.append(q)
    return qs


def first_appearance(q):
    V = []
    for R in q.relations:
        for a in R.attrs:
            if a not in V:
                V.append(a)
    return V


@pytest.mark.parametrize("q", tiny_cyclic(), ids=lambda q: f"{q.name}{id(q) % 997}")
def test_cyclic_queries_match_nested_loops(q):
    """Queries whose relation order gives no join tree (4- and 5-cycles, two
    triangles, all pairs of four attributes, three-key relations, a cycle
    with a leaf): every row combination agreeing on all shared attributes,
    ordered by V (attributes by first appearance), then the row ids; the
    columns and the GFJS levels by their definitions."""
    pl = O.plan(q)
    assert pl.cyclic and pl.kind == "cyclic"
    assert pl.V == first_appearance(q)
    bf = canonical(q, brute_force(q), pl.V)
    assert O.count(q).total == len(bf)
    j = O.join(q)
    assert [tuple(t) for t in j.rowids.tolist()] == [tuple(t) for t in bf]
    cols = O.columns(q, j.rowids)
    for i, t in enumerate(bf[:40]):
        assert [int(cols[v][i]) for v in range(len(pl.V))] == [value_of(q, t, a) for a in pl.V]
    lv = O.gfjs_levels(q, j.rowids)
    ref = levels_by_definition(q, bf, pl.V)
    for l in range(len(pl.V)):
        assert [list(x) for x in zip(lv[l].value.tolist(), lv[l].freq.tolist(),
                                     lv[l].offset.tolist())] == ref[l]


@pytest.mark.parametrize("shape,seed,s", [("square", 0, 0.0), ("square", 1, 1.2), ("pentagon", 2, 0.7),
                                          ("pentagon", 3, 0.0)])
def test_cycle_size_is_the_trace_of_the_count_matrices(shape, seed, s):
    # an L-cycle R_i(A_i, A_i+1 mod L): |Q| = sum over (a_0..a_L-1) of
    # prod_i n_i(a_i, a_i+1) = trace(M_0 ... M_L-1), M_i the pair-count
    # matrices: a library matrix product, independent of the oracle's joins
    d = 9 + seed
    q = G.cyclic_query(9200 + seed, shape, [200 + 37 * i for i in range(5)][:len(G.CYCLIC_SHAPES[shape])],
                       domain=d, s=s)
    P = np.eye(d, dtype=np.int64)
    for R in q.relations:
        m = np.zeros((d, d), np.int64)
        np.add.at(m, (R.keys[0].astype(np.int64), R.keys[1].astype(np.int64)), 1)
        P = P @ m
    assert O.count(q).total == int(np.trace(P))


def test_cyclic_all_equal_keys_give_the_product():
    for shape in G.CYCLIC_SHAPES:
        rows = [2 + i for i in range(len(G.CYCLIC_SHAPES[shape]))]
        q = G.cyclic_query(1, shape, rows, domain=1)
        assert O.count(q).total == int(np.prod(rows)), shape


@pytest.mark.parametrize("seed", range(6))
def test_general_cyclic_path_equals_the_triangle_path(seed):
    # the 3-cycle has its own path (two equi-joins); the general cascade,
    # given the same query, gives the same rows in the same order
    q = G.triangle_query(9300 + seed, [40, 50, 30], domain=4 + seed % 3, s=0.5 * (seed % 3))
    pl = O.cyclic_plan(q)
    assert pl.V == O.plan(q).V
    assert np.array_equal(O._cyclic_rowids(q, pl), O.join(q).rowids)


def test_queries_without_a_shared_attribute_are_rejected():
    # a relation sharing no attribute with those before it makes a cross
    # product, not an equi-join; early projection of a cyclic query is not
    # supported
    a = np.array([0, 1], np.int32)
    cross = G.Query("cross", [G.Relation("R", [0, 1], [a, a]), G.Relation("S", [2, 3], [a, a])])
    with pytest.raises(O.NotAcyclic):
        O.plan(cross)
    sq = G.cyclic_query(2, "pendant", 4, domain=2)
    with pytest.raises(O.NotAcyclic):
        O.plan(sq, drop=[5])


def test_plan_of_branching_tree():
    z = np.zeros(1, np.int32)
    # R0(A,B) root; R1(B,C) under R0; R2(A,D) under R0; R3(C,E) under R1
    q = G.Query("tree", [G.Relation("R0", [0, 1], [z, z]), G.Relation("R1", [1, 2], [z, z]),
                         G.Relation("R2", [0, 3], [z, z]), G.Relation("R3", [2, 4], [z, z])])
    pl = O.plan(q)
    assert pl.parent == [-1, 0, 0, 1]
    assert pl.preorder == [0, 1, 3, 2]
    assert pl.V == [0, 1, 2, 4, 3]


# ------------------------------------------------------------------ closed forms

def _all_equal_star(sizes, value=7):
    rels = [G.Relation(f"R{i}", [0], [np.full(n, value, np.int32)]) for i, n in enumerate(sizes)]
    return G.Query("allequal", rels)


def test_all_keys_equal_gives_product():
    sizes = [3, 4, 5, 6]
    c = O.count(_all_equal_star(sizes))
    assert c.total == 3 * 4 * 5 * 6


def test_empty_table_gives_zero():
    q = G.chain3_uniform(rows=100, end_domain=10, mid_domain=5)
    q.relations[1] = G.Relation("R2", [1, 2], [np.zeros(0, np.int32)] * 2, [np.zeros(0, np.int32)])
    assert O.count(q).total == 0
    q0 = G.chain3_uniform(rows=100, end_domain=10, mid_domain=5)
    q0.relations[0] = G.Relation("R1", [0, 1], [np.zeros(0, np.int32)] * 2, [np.zeros(0, np.int32)])
    assert O.count(q0).total == 0


def test_primary_key_foreign_key_chain_counts_surviving_rows():
    rng = np.random.default_rng(5)
    fact_fk = rng.integers(0, 200, size=5000, dtype=np.int32)
    dim_pk = np.arange(0, 200, 2, dtype=np.int32)          # every other key exists
    rng.shuffle(dim_pk)
    q = G.Query("pkfk", [G.Relation("F", [0], [fact_fk]), G.Relation("D", [0], [dim_pk])])
    assert O.count(q).total == int((fact_fk % 2 == 0).sum())


def test_uniform_chain_expected_size():
    # E|Q| = n^3 / (|dom B| |dom C|) = 10^12 / 10^6 for the uniform 3-chain
    c = O.count(G.chain3_uniform())
    assert abs(c.total - 10**6) < 0.05 * 10**6


def test_agm_bound_holds_on_chains():
    # chain R1(A,B) R2(B,C) R3(C,D) over sets (the bound of Eq. 1 is for
    # relations without duplicate rows): lambda = (1, 0, 1) covers every
    # attribute, so |Q| <= |R1| |R3|
    for seed in range(20):
        q = G.chain_query("c", [30, 40, 50], [6, 3, 3, 6], [0.5] * 4, None, seed)
        for i, R in enumerate(q.relations):
            u = np.unique(np.stack(R.keys, axis=1), axis=0)
            q.relations[i] = G.Relation(R.name, R.attrs, [u[:, 0].copy(), u[:, 1].copy()])
        n1, n3 = q.relations[0].n_rows, q.relations[2].n_rows
        assert O.count(q).total <= n1 * n3


# ------------------------------------------------------------------ 2^64 boundary

def test_largest_exact_count_is_two_pow_64_minus_2():
    sizes = [2, 7, 7, 73, 127, 337, 92737, 649657]        # product = 2^64 - 2
    c = O.count(_all_equal_star(sizes))
    assert c.total == (1 << 64) - 2 and not c.overflow


def test_two_pow_64_minus_1_reports_overflow():
    sizes = [3, 5, 17, 257, 641, 65537, 6700417]           # product = 2^64 - 1
    c = O.count(_all_equal_star(sizes))
    assert c.overflow and c.total == CAP


def test_beyond_two_pow_64_reports_overflow():
    c = O.count(_all_equal_star([256] * 9))               # 2^72
    assert c.overflow and c.total == CAP


def test_dead_branch_never_reports_overflow():
    # R0(A) holds only A=1; the subtree under A=2 has 256^8 = 2^64 ways
    rels = [G.Relation("R0", [0], [np.array([1, 1, 1], np.int32)])]
    rels.append(G.Relation("R1", [0, 1], [np.full(256, 2, np.int32), np.zeros(256, np.int32)]))
    for i in range(2, 9):
        rels.append(G.Relation(f"R{i}", [1], [np.zeros(256, np.int32)]))
    rels.append(G.Relation("R9", [0], [np.array([1, 2], np.int32)]))
    q = G.Query("dead", rels)
    c = O.count(q, rows=True)
    assert c.total == 0 and not c.overflow
    assert all(int(m.max(initial=0)) == 0 for m in c.mult)


def test_aligned_zipf_chain_overflows():
    # heavy hitters that line up across tables (key = rank): the 5-chain's
    # size is far above 2^64 (Section 8 overflow case), at reduced scale
    q = G.chain5_zipf(rows=10**6, domain=10**5, aligned=True)
    c = O.count(q)
    assert c.overflow
    # the same tables with per-column permutations stay exact
    q2 = G.chain5_zipf(rows=10**5, domain=10**5)
    c2 = O.count(q2)
    assert not c2.overflow and 0 < c2.total < CAP


# ------------------------------------------------------------------ wider shapes

def _shape_queries():
    qs = []
    for seed in range(40):
        n_rel = 2 + seed % 4
        qs.append(G.random_tree_query(500 + seed, n_rel, max_rows=5 if n_rel <= 3 else 4,
                                      domain=3, max_new=2, min_rows=1, max_shared=3,
                                      spread=(seed % 3) * 600_000_007 % 2_000_000_000 // 3))
    return qs


@pytest.mark.parametrize("q", _shape_queries(), ids=lambda q: q.name)
def test_oracle_matches_nested_loops_multi_attribute_separators(q):
    pl = O.plan(q)
    bf = canonical(q, brute_force(q), pl.V)
    c = O.count(q)
    assert c.total == len(bf)
    if bf:
        assert [tuple(t) for t in O.join(q).rowids.tolist()] == [tuple(t) for t in bf]


def _int32_end_queries():
    qs = []
    for seed in range(30):
        n_rel = 1 + seed % 4
        base = G.random_tree_query(2100 + seed, n_rel, max_rows=5 if n_rel <= 2 else 4,
                                   domain=3, max_new=2, min_rows=1, max_shared=2)
        qs.append(G.extreme_keys(base, seed))
    return qs


@pytest.mark.parametrize("q", _int32_end_queries(), ids=lambda q: q.name)
def test_oracle_matches_nested_loops_at_the_int32_ends(q):
    # keys at INT32_MIN, INT32_MAX and around zero: the result is ordered by
    # the signed values (no wrap in a key difference or a packed word) and
    # the levels' runs follow that order
    pl = O.plan(q)
    bf = canonical(q, brute_force(q), pl.V)
    c = O.count(q, rows=True)
    assert c.total == len(bf)
    if not bf:
        return
    j = O.join(q)
    assert [tuple(t) for t in j.rowids.tolist()] == [tuple(t) for t in bf]
    lv = O.gfjs_levels(q, j.rowids)
    ref = levels_by_definition(q, bf, pl.V)
    for l in range(len(pl.V)):
        assert [list(x) for x in zip(lv[l].value.tolist(), lv[l].freq.tolist(),
                                     lv[l].offset.tolist())] == ref[l]


def test_duplicated_tables_multiply_the_join_size():
    base = G.chain_sensitivity(rows=2000, domain=500, hops=3)
    assert O.count(G.duplicate_rows(base)).total == 8 * O.count(base).total
    assert O.count(G.duplicate_rows(base, 3)).total == 27 * O.count(base).total
