"""Seeded synthetic relations for n-way equi-join workloads.

This module only draws random numbers and lays them out as columnar tables.
It holds none of the join method's arithmetic, so that both the CPU oracle
and the CUDA path can take identical inputs from it.

The paper evaluates on JOB, TPC-H and lastFM queries (Section 4, "Data" and
"Queries"); those datasets are not used here.  The generators below produce
stand-ins with the shapes the paper's many-to-many workloads have: chain and
star joins whose join attributes are skewed (Zipf) or uniform, tables with
duplicate key tuples (bag semantics, Figure 1), and key values that die
between joins (unneeded intermediate results, Section 1.1).

Conventions
-----------
* A relation is a set of int32 key columns, each bound to an attribute id,
  plus payload columns (int32 or int64) that are carried through the join.
* Two relations join on every attribute id they share.
* A query lists its relations with the root first.
* Zipf(s, D): rank r in [0, D) drawn with probability proportional to
  (r+1)^-s by inverse-CDF lookup; s = 0 is uniform.  The key value is a
  seeded random permutation of the rank, drawn separately for every
  (relation, column), so heavy hitters of different tables do not line up.
  ``aligned=True`` skips the permutation (key = rank), which makes heavy
  hitters coincide and is used to build joins whose size exceeds 2^64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20261203


@dataclass
class Relation:
    name: str
    attrs: list            # attribute id per key column
    keys: list             # np.int32[n] per key column
    payloads: list = field(default_factory=list)   # np.int32[n] or np.int64[n]

    @property
    def n_rows(self) -> int:
        if self.keys:
            return int(self.keys[0].shape[0])
        if self.payloads:
            return int(self.payloads[0].shape[0])
        return 0


@dataclass
class Query:
    name: str
    relations: list        # relations[0] is the root
    attr_names: dict = field(default_factory=dict)

    @property
    def n_rows_total(self) -> int:
        return sum(r.n_rows for r in self.relations)


_CDF_CACHE: dict = {}


def _zipf_cdf(s: float, D: int) -> np.ndarray:
    key = (float(s), int(D))
    cdf = _CDF_CACHE.get(key)
    if cdf is None:
        p = np.arange(1, D + 1, dtype=np.float64) ** (-float(s))
        cdf = np.cumsum(p)
        cdf /= cdf[-1]
        _CDF_CACHE.clear()
        _CDF_CACHE[key] = cdf
    return cdf


def zipf_ranks(rng: np.random.Generator, n: int, s: float, D: int) -> np.ndarray:
    """n ranks in [0, D) with P(r) proportional to (r+1)^-s (uniform if s == 0)."""
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    if s == 0.0:
        return rng.integers(0, D, size=n, dtype=np.int64)
    cdf = _zipf_cdf(s, D)
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="right")
    np.minimum(r, D - 1, out=r)
    return r


def zipf_keys(rng: np.random.Generator, n: int, s: float, D: int,
              aligned: bool = False) -> np.ndarray:
    r = zipf_ranks(rng, n, s, D)
    if aligned or s == 0.0:
        return r.astype(np.int32)
    perm = rng.permutation(D).astype(np.int32)
    return perm[r]


def _payload(rng: np.random.Generator, n: int, dtype) -> np.ndarray:
    info = np.iinfo(dtype)
    return rng.integers(info.min, info.max, size=n, dtype=dtype, endpoint=True)


def chain_query(name: str, rows, domains, s, payload_dtype, seed: int,
                aligned: bool = False) -> Query:
    """Chain R_1(K_0,K_1) join R_2(K_1,K_2) join ... join R_k(K_{k-1},K_k).

    rows[i] is |R_{i+1}|; domains[j] and s[j] are the domain size and Zipf
    exponent of attribute K_j (len k+1).
    """
    k = len(rows)
    assert len(domains) == k + 1 and len(s) == k + 1
    rng = np.random.default_rng(seed)
    rels = []
    for i in range(k):
        n = int(rows[i])
        cols = [zipf_keys(rng, n, s[i], int(domains[i]), aligned),
                zipf_keys(rng, n, s[i + 1], int(domains[i + 1]), aligned)]
        pays = [_payload(rng, n, payload_dtype)] if payload_dtype is not None else []
        rels.append(Relation(f"R{i + 1}", [i, i + 1], cols, pays))
    names = {j: f"K{j}" for j in range(k + 1)}
    return Query(name, rels, names)


def chain3_uniform(seed: int = SEED_BASE + 0, rows: int = 10**4,
                   end_domain: int = 10**4, mid_domain: int = 1000) -> Query:
    """R1(A,B) join R2(B,C) join R3(C,D): A, D uniform over [0, end_domain),
    B, C uniform over [0, mid_domain), one int32 payload per table."""
    q = chain_query("chain3_uniform", [rows] * 3,
                    [end_domain, mid_domain, mid_domain, end_domain],
                    [0.0] * 4, np.int32, seed)
    q.attr_names = {0: "A", 1: "B", 2: "C", 3: "D"}
    return q


def chain5_zipf(seed: int = SEED_BASE + 1, rows: int = 10**7, domain: int = 10**6,
                s: float = 1.1, aligned: bool = False) -> Query:
    """R_i(K_{i-1},K_i), i = 1..5, Zipf(s) keys over [0, domain), one int64
    payload per table."""
    return chain_query("chain5_zipf", [rows] * 5, [domain] * 6, [s] * 6,
                       np.int64, seed, aligned)


def triangle_query(seed: int, rows, domain: int, s: float = 0.0, payload_dtype=np.int64,
                   name: str = "triangle") -> Query:
    """The cyclic join R(A,B) join S(B,C) join T(C,A): rows[i] rows per table,
    keys Zipf(s) over [0, domain) (uniform for s = 0), one payload per table."""
    rng = np.random.default_rng(seed)
    rels = []
    for i, (x, y) in enumerate([(0, 1), (1, 2), (2, 0)]):
        n = int(rows[i])
        cols = [zipf_keys(rng, n, s, domain), zipf_keys(rng, n, s, domain)]
        pays = [_payload(rng, n, payload_dtype)] if payload_dtype is not None else []
        rels.append(Relation("RST"[i], [x, y], cols, pays))
    return Query(name, rels, {0: "A", 1: "B", 2: "C"})


# Attribute lists of cyclic query shapes (relations in order; a relation's
# keys are these attributes in this declared order).
CYCLIC_SHAPES = {
    "square": [(0, 1), (1, 2), (2, 3), (3, 0)],                       # 4-cycle
    "pentagon": [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)],             # 5-cycle
    "bowtie": [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)],       # two triangles on C
    "diamond": [(0, 1), (1, 2), (2, 0), (2, 3), (3, 0)],              # triangles sharing A-C
    "k4": [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (1, 3)],           # every pair of 4 attributes
    "wide": [(0, 1, 2), (2, 3), (3, 1, 0)],                           # relations with three keys
    "pendant": [(0, 1), (1, 2), (2, 3), (3, 0), (3, 5)],              # 4-cycle and a leaf
}


def cyclic_query(seed: int, shape: str, rows, domain: int, s: float = 0.0,
                 payload_dtype=np.int64) -> Query:
    """A query of one of CYCLIC_SHAPES: rows[i] rows per relation (an int
    gives every relation that many), keys Zipf(s) over [0, domain) (uniform
    for s = 0), one payload per relation (none if payload_dtype is None)."""
    rng = np.random.default_rng(seed)
    attrs = CYCLIC_SHAPES[shape]
    rows = [rows] * len(attrs) if isinstance(rows, (int, np.integer)) else list(rows)
    rels = []
    for i, at in enumerate(attrs):
        n = int(rows[i])
        cols = [zipf_keys(rng, n, s, domain) for _ in at]
        pays = [_payload(rng, n, payload_dtype)] if payload_dtype is not None else []
        rels.append(Relation(f"R{i}", list(at), cols, pays))
    return Query(shape, rels, {a: "ABCDEF"[a] for at in attrs for a in at})


def star_poisson(seed: int = SEED_BASE + 2, fact_rows: int = 10**8, domain: int = 10**6,
                 n_dims: int = 4, lam: float = 2.0) -> Query:
    """Fact F(K_1..K_n, P) with K_j uniform over [0, domain), joined to
    dimension tables D_j(K_j, P_j) that hold Poisson(lam) copies of every key
    in [0, domain), shuffled.  int64 payloads."""
    rng = np.random.default_rng(seed)
    fk = [rng.integers(0, domain, size=fact_rows, dtype=np.int32) for _ in range(n_dims)]
    fact = Relation("F", list(range(1, n_dims + 1)), fk,
                    [_payload(rng, fact_rows, np.int64)])
    rels = [fact]
    for j in range(1, n_dims + 1):
        reps = rng.poisson(lam, size=domain)
        keys = np.repeat(np.arange(domain, dtype=np.int32), reps)
        rng.shuffle(keys)
        rels.append(Relation(f"D{j}", [j], [keys],
                             [_payload(rng, keys.shape[0], np.int64)]))
    names = {j: f"K{j}" for j in range(1, n_dims + 1)}
    return Query("star_poisson", rels, names)


def batch_queries(seed: int = SEED_BASE + 3, n_queries: int = 4096,
                  min_tables: int = 3, max_tables: int = 6,
                  rows_range=(10**3, 10**6), domain_range=(10**2, 10**5),
                  s_range=(0.0, 1.5)) -> list:
    """Independent chain joins: tables per query uniform in [min,max], rows
    per table and domain per attribute log-uniform, one Zipf exponent per
    query uniform in s_range; int32 keys, no payloads."""
    rng = np.random.default_rng(seed)
    out = []
    lo_r, hi_r = np.log(rows_range[0]), np.log(rows_range[1])
    lo_d, hi_d = np.log(domain_range[0]), np.log(domain_range[1])
    for qi in range(n_queries):
        k = int(rng.integers(min_tables, max_tables + 1))
        rows = np.exp(rng.uniform(lo_r, hi_r, size=k)).astype(np.int64)
        doms = np.exp(rng.uniform(lo_d, hi_d, size=k + 1)).astype(np.int64)
        s = float(rng.uniform(*s_range))
        sub = int(rng.integers(0, 2**62))
        out.append(chain_query(f"batch{qi}", rows, doms, [s] * (k + 1), None, sub))
    return out


def random_tree_query(seed: int, n_rel: int, max_rows: int = 6, domain: int = 3,
                      max_new: int = 2, payload: bool = True, min_rows: int = 0,
                      max_shared: int = 1, spread: int = 0) -> Query:
    """Small random acyclic query: relation j > 0 attaches to a random earlier
    relation, shares 1..max_shared of its attributes, and adds 0..max_new
    attributes of its own.  Values are uniform over a small domain so that
    joins match, repeat and die; spread > 0 maps value v to v * spread - 2^30
    (same join structure, values far apart in the int32 range)."""
    rng = np.random.default_rng(seed)
    next_attr = 0
    rel_attrs = []
    for j in range(n_rel):
        if j == 0:
            na = int(rng.integers(1, max_new + 2))
            attrs = list(range(next_attr, next_attr + na))
            next_attr += na
        else:
            par = int(rng.integers(0, j))
            ns = int(rng.integers(1, min(max_shared, len(rel_attrs[par])) + 1))
            shared = [int(x) for x in rng.choice(rel_attrs[par], size=ns, replace=False)]
            na = int(rng.integers(0, max_new + 1))
            new = list(range(next_attr, next_attr + na))
            next_attr += na
            attrs = shared + new
            rng.shuffle(attrs)
        rel_attrs.append([int(a) for a in attrs])
    rels = []
    for j, attrs in enumerate(rel_attrs):
        n = int(rng.integers(min_rows, max_rows + 1))
        cols = [rng.integers(-1, domain - 1, size=n, dtype=np.int32) for _ in attrs]
        if spread:
            cols = [(c.astype(np.int64) * spread - 2**30).astype(np.int32) for c in cols]
        pays = []
        if payload:
            pays = [_payload(rng, n, np.int32), _payload(rng, n, np.int64)]
        rels.append(Relation(f"T{j}", attrs, cols, pays))
    return Query(f"tree{seed}", rels, {a: f"X{a}" for a in range(next_attr)})


_INT32_ENDS = np.array([-2**31, -2**31 + 1, -1, 0, 2**31 - 2, 2**31 - 1], dtype=np.int64)


def extreme_keys(q: Query, seed: int) -> Query:
    """The same query with every attribute's values mapped one-to-one, by a
    seeded permutation per attribute, onto values at both ends of the int32
    range and around zero (INT32_MIN, INT32_MIN + 1, -1, 0, INT32_MAX - 1,
    INT32_MAX).  Which rows join is unchanged; the sorted order of the result
    is not.  The input's key values must lie in [-1, 4] (random_tree_query
    with domain <= 5)."""
    rng = np.random.default_rng(seed)
    maps = {}
    rels = []
    for R in q.relations:
        cols = []
        for a, k in zip(R.attrs, R.keys):
            if a not in maps:
                maps[a] = rng.permutation(_INT32_ENDS)
            idx = k.astype(np.int64) + 1
            if idx.size and (idx.min() < 0 or idx.max() >= _INT32_ENDS.shape[0]):
                raise ValueError("key values outside [-1, 4]")
            cols.append(maps[a][idx].astype(np.int32))
        rels.append(Relation(R.name, list(R.attrs), cols, list(R.payloads)))
    return Query(q.name + "_ends", rels, dict(q.attr_names))


def batch_queries_torch(seed: int = SEED_BASE + 3, n_queries: int = 4096,
                        min_tables: int = 3, max_tables: int = 6,
                        rows_range=(10**3, 10**6), domain_range=(10**2, 10**5),
                        s_range=(0.0, 1.5), device="cuda"):
    """The batch_queries distribution drawn on a CUDA device with torch (for
    batches of billions of rows).  Returns a list of queries, each a list of
    (attrs, [key tensors]) relations; no payloads."""
    import torch
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lo_r, hi_r = np.log(rows_range[0]), np.log(rows_range[1])
    lo_d, hi_d = np.log(domain_range[0]), np.log(domain_range[1])
    cdfs = {}

    def keys(n, s, D):
        if s == 0.0:
            return torch.randint(0, D, (n,), generator=g, device=device, dtype=torch.int32)
        cdf = cdfs.get((s, D))
        if cdf is None:
            p = torch.arange(1, D + 1, device=device, dtype=torch.float64) ** (-s)
            cdf = torch.cumsum(p, 0)
            cdf /= cdf[-1].clone()
            cdfs.clear()
            cdfs[(s, D)] = cdf
        u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
        r = torch.searchsorted(cdf, u, right=True).clamp_(max=D - 1)
        perm = torch.randperm(D, generator=g, device=device)
        return perm[r].to(torch.int32)

    out = []
    for _ in range(n_queries):
        if n_queries == 0:
            break
        k = int(rng.integers(min_tables, max_tables + 1))
        rows = np.exp(rng.uniform(lo_r, hi_r, size=k)).astype(np.int64)
        doms = np.exp(rng.uniform(lo_d, hi_d, size=k + 1)).astype(np.int64)
        s = float(rng.uniform(*s_range))
        rels = []
        for i in range(k):
            n = int(rows[i])
            rels.append(([i, i + 1], [keys(n, s, int(doms[i])), keys(n, s, int(doms[i + 1]))]))
        out.append(rels)
    return out


def chain_zipf_torch(seed: int, tables: int = 4, rows: int = 10**7, domain: int = 10**6,
                     s: float = 1.1, device="cuda"):
    """A chain R_i(K_{i-1}, K_i) with Zipf(s) keys over [0, domain), permuted
    per (relation, column), drawn on a CUDA device; same layout as
    batch_queries_torch (list of (attrs, [key tensors]))."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    p = torch.arange(1, domain + 1, device=device, dtype=torch.float64) ** (-s)
    cdf = torch.cumsum(p, 0)
    cdf /= cdf[-1].clone()

    def keys():
        u = torch.rand(rows, generator=g, device=device, dtype=torch.float64)
        r = torch.searchsorted(cdf, u, right=True).clamp_(max=domain - 1)
        return torch.randperm(domain, generator=g, device=device)[r].to(torch.int32)

    return [([i, i + 1], [keys(), keys()]) for i in range(tables)]


def duplicate_rows(query: Query, times: int = 2) -> Query:
    """Every relation with each row repeated `times` times (the "_dup" form of
    the sensitivity study, Section 4.2): the join size grows by times^k while
    the distinct key tuples stay the same."""
    rels = []
    for R in query.relations:
        rels.append(Relation(R.name + "_dup", list(R.attrs),
                             [np.tile(k, times) for k in R.keys],
                             [np.tile(p, times) for p in R.payloads]))
    return Query(query.name + "_dup", rels, dict(query.attr_names))


def chain_sensitivity(seed: int = SEED_BASE + 7, rows: int = 10**6, domain: int = 10**5,
                      s: float = 1.1, hops: int = 3) -> Query:
    """The base chain of the sensitivity study: `hops` tables R_i(K_{i-1}, K_i)
    with Zipf(s) keys (the shape of a user-item-friend chain); hops + 1 adds
    one join and with it more unneeded intermediate results (Section 4.2)."""
    return chain_query(f"sens{hops}", [rows] * hops, [domain] * (hops + 1), [s] * (hops + 1),
                       np.int64, seed)
