"""CPU oracle for acyclic n-way equi-joins (Graphical Join, arXiv 2206.10435).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path: it plans the join tree itself, and its arithmetic lives in
``gj_oracle.c`` (counting pass, cascade of binary hash joins, canonical
sort) and in the plain numpy definitions below (summary levels, per-tuple
multiplicities, materialised columns).

Readings of the paper that this oracle fixes:

* Bag semantics: duplicate rows each count (Figure 1 / Figure 2: 32 result
  tuples from tables with repeated rows).
* Join tree: relation 0 is the root; relation j > 0 hangs under the first
  earlier relation that holds every attribute j shares with relations
  0..j-1 (its separator).  No such relation means the order does not give a
  join tree and the query is rejected.
* Variable order V (the order of the summary's columns, Section 3.5): a
  preorder walk of the join tree from the root, children in index order;
  each relation contributes the attributes its parent lacks, in declared
  column order.  For the running example this gives A, B, C, D (root A).
* Canonical result order (Def. 1 sorts by all columns): ascending signed
  int32 values of V, ties broken by the original row indices r_1..r_k.
* Summary level l (Def. 1, Algorithm 4's per-level emission): one run per
  distinct prefix (v_0..v_l) of the canonically ordered result, holding the
  value v_l, its frequency and the offset of the run.  Runs of frequency 0
  do not exist (Section 3.3: entries below 1 are dropped).
* Counts are exact below 2^64 - 1; that value marks a clamped count, and a
  join whose size reaches it is reported as overflowing.
* The cyclic 3-way join R0(A,B), R1(B,C), R2(C,A) (any column order): V is
  R0's columns in declared order, then C; the result (the same plain
  definition: every row combination agreeing on all shared attributes) is
  computed by sort-based equi-joins R0 |><| R1 on B, then with R2 on (C, A),
  and put in canonical order by a sort.
* Any other query whose relation order gives no join tree (Sections 3.2.1
  and 3.4 answer it over a junction tree): when every relation after the
  first shares an attribute with the relations before it, V is the
  attributes in order of first appearance (relation 0's columns in declared
  order, then each relation's new attributes in declared column order); the
  result is again every row combination agreeing on all shared attributes,
  built by a cascade of sort-based equi-joins, relation j joined on every
  attribute it shares with relations 0..j-1, then sorted canonically.
* Early projection (Section 3.7): a dropped attribute is deleted from V.
  The result is the same bag of row-id tuples, its columns are the
  remaining V attributes and the payloads, and its rows are ordered by the
  remaining V values, then the row ids.  Only attributes held by exactly
  one relation can be dropped (a shared one would need the potential join).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
CAP = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile gj_oracle.c into oracle/_build/liboracle.so (plain gcc)."""
    src = os.path.join(_HERE, "gj_oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_count.restype = ctypes.c_int
        _lib.orc_join.restype = ctypes.c_int64
    return _lib


class _Rel(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_keys", ctypes.c_int32),
                ("key", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)))]


class _Query(ctypes.Structure):
    _fields_ = [("n_rel", ctypes.c_int32), ("rel", ctypes.POINTER(_Rel)),
                ("parent", ctypes.POINTER(ctypes.c_int32)),
                ("sep_w", ctypes.POINTER(ctypes.c_int32)),
                ("sep_cj", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                ("sep_cp", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                ("n_vars", ctypes.c_int32),
                ("var_rel", ctypes.POINTER(ctypes.c_int32)),
                ("var_col", ctypes.POINTER(ctypes.c_int32))]


class NotAcyclic(ValueError):
    pass


@dataclass
class Plan:
    parent: list       # parent relation per relation (-1 for the root)
    sep: list          # separator attribute ids per relation (empty for root)
    preorder: list     # relation indices in preorder
    V: list            # attribute ids in summary-column order
    var_rel: list      # relation that introduces V[i]
    var_col: list      # its column there
    cyclic: bool = False   # no join tree: the 3-cycle, or a general cyclic query
    kind: str = "tree"     # "tree", "triangle" (R0(A,B), R1(B,C), R2(C,A)) or "cyclic"


def _triangle(rels):
    """(ab, bc, ca) if the relations form the cycle R0(A,B), R1(B,C), R2(C,A)."""
    if len(rels) != 3 or any(len(R.attrs) != 2 or R.attrs[0] == R.attrs[1] for R in rels):
        return None

    def shared(x, y):
        s = [a for a in rels[x].attrs if a in rels[y].attrs]
        return s[0] if len(s) == 1 else None
    ab, bc, ca = shared(0, 1), shared(1, 2), shared(2, 0)
    if None in (ab, bc, ca) or len({ab, bc, ca}) != 3:
        return None
    return ab, bc, ca


def plan(query, drop=()) -> Plan:
    rels = query.relations
    tri = None if drop else _triangle(rels)
    if tri:
        ab, bc, ca = tri
        return Plan([-1, 0, 1], [[], [ab], [bc, ca]], [0, 1, 2], list(rels[0].attrs) + [bc],
                    [0, 0, 1], [0, 1, rels[1].attrs.index(bc)], cyclic=True, kind="triangle")
    drop = set(drop)
    for a in drop:
        if sum(R.attrs.count(a) for R in rels) != 1:
            raise ValueError(f"attribute {a} is not held by exactly one relation")
    k = len(rels)
    parent, sep = [-1], [[]]
    seen = set(rels[0].attrs) if k else set()
    for j in range(1, k):
        shared = [a for a in rels[j].attrs if a in seen]
        if not shared:
            raise NotAcyclic(f"relation {j} shares no attribute with relations before it")
        p = next((i for i in range(j) if set(shared) <= set(rels[i].attrs)), None)
        if p is None:
            if drop:
                raise NotAcyclic(f"relation {j}: no earlier relation holds all of {shared}")
            return cyclic_plan(query)
        parent.append(p)
        sep.append(shared)
        seen.update(rels[j].attrs)
    order = []
    stack = [0] if k else []
    while stack:
        t = stack.pop()
        order.append(t)
        stack.extend(reversed([c for c in range(k) if parent[c] == t]))
    V, var_rel, var_col = [], [], []
    for t in order:
        for c, a in enumerate(rels[t].attrs):
            if a not in V and a not in drop:
                V.append(a)
                var_rel.append(t)
                var_col.append(c)
    return Plan(parent, sep, order, V, var_rel, var_col)


def cyclic_plan(query) -> Plan:
    """The plan of a query whose relation order gives no join tree: V by
    first appearance; sep[j] = every attribute relation j shares with
    relations 0..j-1 (it must share one); parent[j] = the first earlier
    relation sharing one of them."""
    rels = query.relations
    parent, sep, seen = [-1], [[]], set(rels[0].attrs) if rels else set()
    for j in range(1, len(rels)):
        shared = [a for a in rels[j].attrs if a in seen]
        if not shared:
            raise NotAcyclic(f"relation {j} shares no attribute with relations before it")
        parent.append(next(i for i in range(j) if set(shared) & set(rels[i].attrs)))
        sep.append(shared)
        seen.update(rels[j].attrs)
    V, var_rel, var_col = [], [], []
    for t, R in enumerate(rels):
        for c, a in enumerate(R.attrs):
            if a not in V:
                V.append(a)
                var_rel.append(t)
                var_col.append(c)
    return Plan(parent, sep, list(range(len(rels))), V, var_rel, var_col, cyclic=True, kind="cyclic")


def _cyclic_rowids(query, pl) -> np.ndarray:
    """Row-id tuples of a query by the plain definition (every combination
    of rows agreeing on all shared attributes), in canonical order: a
    cascade of sort-based equi-joins, relation j joined on all the
    attributes it shares with relations 0..j-1, then one sort."""
    rels = query.relations
    col = lambda R, a: np.asarray(R.keys[R.attrs.index(a)], dtype=np.int64)
    t = np.arange(rels[0].n_rows, dtype=np.int64).reshape(-1, 1)
    holder = {a: 0 for a in rels[0].attrs}          # first relation holding an attribute
    for j in range(1, len(rels)):
        R = rels[j]
        shared = pl.sep[j]
        left = np.stack([col(rels[holder[a]], a)[t[:, holder[a]]] for a in shared], axis=1)
        right = np.stack([col(R, a) for a in shared], axis=1)
        # shared-value tuples of both sides numbered alike, then one equi-join
        both = np.concatenate([left, right]) if left.shape[0] + right.shape[0] else left
        if both.shape[0]:
            _, ids = np.unique(both, axis=0, return_inverse=True)
            ids = ids.reshape(-1)
        else:
            ids = np.zeros(0, np.int64)
        li, ri = _equi_join(ids[:left.shape[0]], ids[left.shape[0]:])
        t = np.concatenate([t[li], ri.reshape(-1, 1)], axis=1)
        for a in R.attrs:
            holder.setdefault(a, j)
    keys = [t[:, c] for c in reversed(range(t.shape[1]))]
    keys += [col(rels[r], a)[t[:, r]] for r, a in zip(reversed(pl.var_rel), reversed(pl.V))]
    order = np.lexsort(keys) if t.shape[0] else np.zeros(0, np.int64)
    return t[order].astype(np.int32)


class _Marshal:
    """Keeps the ctypes views of one query alive."""

    def __init__(self, query, pl: Plan):
        rels = query.relations
        k = len(rels)
        self.keep = []
        self.rels = (_Rel * max(k, 1))()
        for j, R in enumerate(rels):
            cols = [np.ascontiguousarray(c, dtype=np.int32) for c in R.keys]
            self.keep.extend(cols)
            arr = (ctypes.POINTER(ctypes.c_int32) * max(len(cols), 1))(
                *[c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for c in cols])
            self.keep.append(arr)
            self.rels[j].n_rows = R.n_rows
            self.rels[j].n_keys = len(cols)
            self.rels[j].key = ctypes.cast(arr, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)))

        def i32(xs):
            a = np.ascontiguousarray(np.asarray(xs, dtype=np.int32).reshape(-1))
            if a.size == 0:
                a = np.zeros(1, dtype=np.int32)
            self.keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

        cj, cp = [], []
        for j in range(k):
            cj.append(i32([rels[j].attrs.index(a) for a in pl.sep[j]]))
            cp.append(i32([rels[pl.parent[j]].attrs.index(a) for a in pl.sep[j]]
                          if j > 0 else []))
        cja = (ctypes.POINTER(ctypes.c_int32) * max(k, 1))(*cj)
        cpa = (ctypes.POINTER(ctypes.c_int32) * max(k, 1))(*cp)
        self.keep += [cja, cpa]
        self.q = _Query(k, self.rels, i32(pl.parent), i32([len(s) for s in pl.sep]),
                        ctypes.cast(cja, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                        ctypes.cast(cpa, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                        len(pl.V), i32(pl.var_rel), i32(pl.var_col))


@dataclass
class Counts:
    total: int                 # |Q|, or CAP when clamped
    overflow: bool
    up: list = None            # per relation, uint64 per row
    down: list = None
    mult: list = None          # per relation, result tuples each row is in


def _equi_join(left_keys, right_keys):
    """All (i, j) with left_keys[i] == right_keys[j], i ascending, j
    ascending within i (a sort of the right side, then ranges)."""
    order = np.argsort(right_keys, kind="stable")
    rs = right_keys[order]
    lo = np.searchsorted(rs, left_keys, "left")
    hi = np.searchsorted(rs, left_keys, "right")
    cnt = (hi - lo).astype(np.int64)
    li = np.repeat(np.arange(left_keys.shape[0], dtype=np.int64), cnt)
    first = np.repeat(lo - (np.cumsum(cnt) - cnt), cnt)
    return li, order[first + np.arange(li.shape[0], dtype=np.int64)]


def _triangle_rowids(query, pl) -> np.ndarray:
    """Row-id triples of the cyclic join, in canonical order."""
    R0, R1, R2 = query.relations
    ab, (bc, ca) = pl.sep[1][0], pl.sep[2]
    col = lambda R, a: np.asarray(R.keys[R.attrs.index(a)], dtype=np.int64)
    i0, i1 = _equi_join(col(R0, ab), col(R1, ab))
    pair_ca = (col(R1, bc)[i1] << 32) | (col(R0, ca)[i0] & 0xFFFFFFFF)
    r2_ca = (col(R2, bc) << 32) | (col(R2, ca) & 0xFFFFFFFF)
    p, i2 = _equi_join(pair_ca, r2_ca)
    t = np.stack([i0[p], i1[p], i2], axis=1).astype(np.int64)
    v0 = np.asarray(R0.keys[0])[t[:, 0]]
    v1 = np.asarray(R0.keys[1])[t[:, 0]]
    vc = col(R1, bc)[t[:, 1]]
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0], vc, v1, v0))
    return t[order].astype(np.int32)


def count(query, rows: bool = False) -> Counts:
    """Join size by the row-level counting pass (and per-row multiplicities)."""
    pl = plan(query)
    if pl.cyclic:
        if rows:
            raise NotImplementedError("per-row multiplicities of the cyclic join")
        t = _triangle_rowids(query, pl) if pl.kind == "triangle" else _cyclic_rowids(query, pl)
        return Counts(int(t.shape[0]), False)
    lib = _load()
    m = _Marshal(query, pl)
    k = len(query.relations)
    up = [np.zeros(max(R.n_rows, 1), dtype=np.uint64) for R in query.relations]
    down = [np.zeros(max(R.n_rows, 1), dtype=np.uint64) for R in query.relations] if rows else None
    mult = [np.zeros(max(R.n_rows, 1), dtype=np.uint64) for R in query.relations] if rows else None

    def ptrs(arrs):
        if arrs is None:
            return None
        return (ctypes.POINTER(ctypes.c_uint64) * k)(
            *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) for a in arrs])

    total = ctypes.c_uint64(0)
    rc = lib.orc_count(ctypes.byref(m.q), ptrs(up), ptrs(down), ptrs(mult), ctypes.byref(total))
    if rc < 0:
        raise MemoryError("oracle counting pass ran out of memory")
    trim = lambda arrs: None if arrs is None else [a[:R.n_rows] for a, R in zip(arrs, query.relations)]
    return Counts(int(total.value), rc == 1, trim(up), trim(down), trim(mult))


@dataclass
class Joined:
    rowids: np.ndarray         # int32[|Q|, k], canonical order
    intermediate: list         # size of the cascade after joining 0..j


def join(query, max_tuples: int = 50_000_000, drop=()) -> Joined:
    """Materialise the join (cascade of hash joins + canonical sort, by the
    V of the projection when attributes are dropped)."""
    pl = plan(query, drop)
    if pl.cyclic:
        t = _triangle_rowids(query, pl) if pl.kind == "triangle" else _cyclic_rowids(query, pl)
        if t.shape[0] > max_tuples:
            raise ValueError(f"join result too large to materialise ({t.shape[0]} tuples)")
        return Joined(t, [])
    lib = _load()
    m = _Marshal(query, pl)
    k = len(query.relations)
    c = count(query)
    if c.overflow or c.total > max_tuples:
        raise ValueError(f"join result too large to materialise ({c.total} tuples)")
    out = np.zeros((max(c.total, 1), k), dtype=np.int32)
    inter = np.zeros(k, dtype=np.int64)
    n = lib.orc_join(ctypes.byref(m.q), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     ctypes.c_int64(c.total), ctypes.c_int64(max_tuples),
                     inter.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if n == -2:
        raise ValueError("an intermediate result of the cascade exceeds max_tuples")
    if n < 0:
        raise MemoryError("oracle join ran out of memory")
    assert n == c.total, (n, c.total)
    return Joined(out[:n], [int(x) for x in inter])


def columns(query, rowids: np.ndarray, drop=()) -> list:
    """Materialised columns: the V attributes (int32), then every
    relation's payloads in relation order (Section 3.6: the flat result)."""
    pl = plan(query, drop)
    cols = []
    for t, c in zip(pl.var_rel, pl.var_col):
        cols.append(query.relations[t].keys[c][rowids[:, t]])
    for j, R in enumerate(query.relations):
        for p in R.payloads:
            cols.append(p[rowids[:, j]])
    return cols


@dataclass
class Level:
    value: np.ndarray          # int32 value of V[l] per run
    freq: np.ndarray           # uint64 run length
    offset: np.ndarray         # uint64 first result row of the run


def gfjs_levels(query, rowids: np.ndarray, drop=()) -> list:
    """Summary levels of the canonically ordered result: level l holds one
    run per distinct prefix (v_0..v_l) (Def. 1, Algorithm 4)."""
    pl = plan(query, drop)
    n = rowids.shape[0]
    vcols = columns(query, rowids, drop)[:len(pl.V)]
    levels = []
    change = np.zeros(n, dtype=bool)
    if n:
        change[0] = True
    for l in range(len(pl.V)):
        if n > 1:
            change[1:] |= vcols[l][1:] != vcols[l][:-1]
        starts = np.flatnonzero(change)
        ends = np.append(starts[1:], n)
        levels.append(Level(vcols[l][starts].astype(np.int32),
                            (ends - starts).astype(np.uint64), starts.astype(np.uint64)))
    return levels


def _distinct_tuples(R):
    """Distinct key tuples of a relation, sorted ascending in declared column
    order, and the index of every row's tuple among them."""
    if R.n_rows == 0:
        return np.zeros((0, len(R.keys)), np.int32), np.zeros(0, np.int64)
    keys = np.stack(R.keys, axis=1)
    allk, inv = np.unique(keys, axis=0, return_inverse=True)
    return allk, inv.reshape(-1)


def group_mult_from_rows(query, rowids: np.ndarray) -> list:
    """Per relation: distinct key tuples and the number of result tuples
    that use each one, counted directly from the materialised result."""
    out = []
    for j, R in enumerate(query.relations):
        allk, inv = _distinct_tuples(R)
        m = np.zeros(allk.shape[0], dtype=np.uint64)
        if rowids.shape[0]:
            np.add.at(m, inv[rowids[:, j]], np.uint64(1))
        out.append((allk, m))
    return out


def group_mult_from_counts(query, c: Counts) -> list:
    """Per relation: distinct key tuples and the summed per-row
    multiplicities of the counting pass (clamped at CAP)."""
    out = []
    for j, R in enumerate(query.relations):
        allk, inv = _distinct_tuples(R)
        mult = c.mult[j]
        if mult.size and (mult == np.uint64(CAP)).any() or c.overflow:
            m = np.zeros(allk.shape[0], dtype=object)
            for i, v in zip(inv.tolist(), mult.tolist()):
                m[i] = min(int(m[i]) + int(v), CAP)
            m = m.astype(np.uint64)
        else:
            m = np.zeros(allk.shape[0], dtype=np.uint64)
            np.add.at(m, inv, mult)
        out.append((allk, m))
    return out
