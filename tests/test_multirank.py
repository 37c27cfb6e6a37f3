"""Multi-rank paths on the CPU: world_size-2 gloo ranks run the partition
and collective code of paper_2206_10435_gb300/partition.py that bench.py
uses under torchrun (one rank per GPU), and the benchmark's reduction."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

SAT = (1 << 64) - 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, world, *args):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _rank_reduce(rank, world, port, out):
    dist = _init(rank, world, port)
    import bench
    # rank r took 100 + 50 r ms and produced 1000 (r + 1) rows
    t, rows = bench.reduce_over_ranks(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
    dist.barrier()
    out.put((rank, t, rows))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_rows():
    assert _spawn(_rank_reduce, 2) == [(0, 150.0, 3000), (1, 150.0, 3000)]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7, "cpu") == (12.5, 7)


def test_row_ranges_partition_the_result():
    from paper_2206_10435_gb300 import partition as P
    for total in (0, 1, 7, 10**6 + 3, (1 << 40) + 5):
        for world in (1, 2, 3, 8):
            rs = [P.row_range(total, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    ws = P.windows(5, 17, 4)
    assert ws == [(5, 4), (9, 4), (13, 4)]
    assert P.windows(3, 3, 4) == []
    with pytest.raises(ValueError):
        P.row_range(10, 2, 2)


def _rank_collectives(rank, world, port, out):
    dist = _init(rank, world, port)
    from paper_2206_10435_gb300 import partition as P
    # per-query results of the rank's block, gathered in query order
    n_total = 7
    lo, hi = P.query_block(n_total, rank, world)
    local = np.array([1000 * q + 1 for q in range(lo, hi)], dtype=np.uint64)
    gathered = P.gather_in_order(dist, local, n_total, rank, world)
    # exact saturating sums: exact just below 2^64 - 1, saturated at and
    # above it, SAT inputs stay SAT, small values exact
    half = np.uint64((1 << 63) - 1)
    vals = {
        0: np.array([5, half, (1 << 63), SAT, 0, (1 << 32) - 1, 1 << 62], dtype=np.uint64),
        1: np.array([7, half, (1 << 63) - 1, 0, 0, (1 << 32) + 1, 1 << 62], dtype=np.uint64),
    }[rank]
    s = P.sum_sat(dist, vals)
    m = P.max_over_ranks(dist, 3.0 + rank)
    out.put((rank, gathered.tolist(), s.tolist(), m))
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_exact_saturating_sum():
    res = _spawn(_rank_collectives, 2)
    want_sum = [12, (1 << 64) - 2, SAT, SAT, 0, 1 << 33, 1 << 63]
    for rank, gathered, s, m in res:
        assert gathered == [1000 * q + 1 for q in range(7)]
        assert s == want_sum, (rank, s)
        assert m == 4.0


def _batch_list():
    from paper_2206_10435_gb300 import datagen as G
    return G.batch_queries(seed=41, n_queries=7, rows_range=(50, 2000), domain_range=(10, 200))


def _rank_batch(rank, world, port, out):
    dist = _init(rank, world, port)
    from oracle import oracle as O
    from paper_2206_10435_gb300 import partition as P
    qs = _batch_list()
    lo, hi = P.query_block(len(qs), rank, world)
    # this rank's block of the global list, counted (the oracle stands in
    # for the GPU path; the split and the gather are what is tested)
    local = np.array([min(int(O.count(q).total), SAT) for q in qs[lo:hi]], dtype=np.uint64)
    gathered = P.gather_in_order(dist, local, len(qs), rank, world)
    out.put((rank, (lo, hi), [int(x) for x in gathered]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_split_a_query_list_and_gather_totals_in_order(world):
    """A list of 7 chain queries split into contiguous blocks over two or
    three ranks: the blocks cover the list once, and every rank gets every
    query's total, in query order."""
    from oracle import oracle as O
    res = _spawn(_rank_batch, world)
    want = [min(int(O.count(q).total), SAT) for q in _batch_list()]
    assert any(w > 0 for w in want)
    blocks = [b for _, b, _ in res]
    assert blocks[0][0] == 0 and blocks[-1][1] == len(want)
    assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
    for _, _, got in res:
        assert got == want


def _rank_rows(rank, world, port, out):
    dist = _init(rank, world, port)
    from oracle import oracle as O
    from paper_2206_10435_gb300 import datagen as G, partition as P
    q = G.chain3_uniform(seed=7, rows=300, end_domain=400, mid_domain=40)
    # every rank holds the same instance; this rank's rows come from the
    # oracle standing in for the GPU path (the partition is what is tested)
    full = O.join(q).rowids
    lo, hi = P.row_range(full.shape[0], rank, world)
    mine = np.concatenate([full[r0:r0 + n] for r0, n in P.windows(lo, hi, 97)] or
                          [full[:0]])
    sizes = torch.tensor([mine.shape[0]], dtype=torch.int64)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes)
    width = full.shape[1]
    pad = max(int(x.item()) for x in all_sizes)
    buf = torch.zeros((pad, width), dtype=torch.int64)
    buf[:mine.shape[0]] = torch.from_numpy(mine.astype(np.int64))
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    joined = np.concatenate([p[:int(n.item())].numpy() for p, n in zip(parts, all_sizes)])
    out.put((rank, bool(np.array_equal(joined, full.astype(np.int64))), full.shape[0]))
    dist.destroy_process_group()


def test_two_gloo_ranks_result_ranges_concatenate_to_the_join():
    res = _spawn(_rank_rows, 2)
    assert all(ok for _, ok, n in res) and res[0][2] > 0


# ---- the row-sharded counting pass (paper_2206_10435_gb300/shard.py) ----

def _plan_parent_sep(query):
    """Join tree by the library's rule: relation j hangs under the first
    earlier relation holding every attribute j shares with relations
    before it; the separator is that (single) shared attribute."""
    parent, sep, seen = [-1], [None], set(query.relations[0].attrs)
    for j, R in enumerate(query.relations[1:], 1):
        shared = [a for a in R.attrs if a in seen]
        assert len(shared) == 1
        parent.append(next(i for i in range(j) if shared[0] in query.relations[i].attrs))
        sep.append(shared[0])
        seen.update(R.attrs)
    return parent, sep


class NumpyShard:
    """A rank's part of the sharded pass computed on the CPU from the
    definitions, row by row (each row is a group of count 1; sums over rows
    equal sums over groups), with Python integers.  It stands in for the
    GPU engine so that the coordination and the collectives run on gloo."""

    def __init__(self, query, rank, world):
        from paper_2206_10435_gb300 import shard as S
        self.parent, self.sep = _plan_parent_sep(query)
        self.attrs = [R.attrs for R in query.relations]
        self.keys = []
        for R in query.relations:
            lo, hi = S.rows_of(R.n_rows, rank, world)
            self.keys.append([k[lo:hi].astype(np.int64) for k in R.keys])
        self.children = {t: [j for j, p in enumerate(self.parent) if p == t]
                         for t in range(len(self.parent))}
        self.local_keys = {}

    def col(self, rel, attr):
        return self.keys[rel][self.attrs[rel].index(attr)]

    def shard_domain(self, rel):
        v = np.concatenate([self.col(rel, self.sep[rel]), self.col(self.parent[rel], self.sep[rel])])
        return (int(v.min()), int(v.max())) if v.size else (1, 0)

    def _at(self, rel, c, msgs):
        vec, lo = msgs[c]
        idx = self.col(rel, self.sep[c]) - lo
        ok = (idx >= 0) & (idx < vec.shape[0])
        out = np.zeros(idx.shape[0], dtype=object)
        out[ok] = [int(x) for x in vec[idx[ok]]]
        return out

    def _prod(self, rel, msgs, skip=None):
        n = self.keys[rel][0].shape[0]
        p = np.ones(n, dtype=object)
        for c in self.children[rel]:
            if c != skip:
                p = p * self._at(rel, c, msgs)
        return p

    @staticmethod
    def _u64(vals):
        return np.array([min(int(v), SAT) for v in vals], dtype=np.uint64)

    def shard_up(self, rel, msgs, lo, length):
        w = self._prod(rel, msgs)
        if self.parent[rel] < 0:
            return self._u64([sum(w)])
        out = [0] * length
        for k, x in zip((self.col(rel, self.sep[rel]) - lo).tolist(), w.tolist()):
            out[k] += x
        return self._u64(out)

    def shard_down(self, rel, down, msgs):
        n = self.keys[rel][0].shape[0]
        if down is None:
            d = np.ones(n, dtype=object)
        else:
            vec, lo = down
            d = np.array([int(vec[k - lo]) for k in self.col(rel, self.sep[rel]).tolist()], dtype=object)
        parts = {}
        for c in self.children[rel]:
            x = d * self._prod(rel, msgs, skip=c)
            vec, lo = msgs[c]
            out = [0] * vec.shape[0]
            for k, v in zip((self.col(rel, self.sep[c]) - lo).tolist(), x.tolist()):
                if 0 <= k < len(out):
                    out[k] += v
            parts[c] = self._u64(out)
        m = d * self._prod(rel, msgs)
        keys = np.stack(self.keys[rel], axis=1) if n else np.zeros((0, len(self.keys[rel])), np.int64)
        uk, inv = np.unique(keys, axis=0, return_inverse=True) if n else (keys, np.zeros(0, np.int64))
        mult = [0] * uk.shape[0]
        for i, v in zip(inv.reshape(-1).tolist(), m.tolist()):
            mult[i] += v
        self.local_keys[rel] = uk
        return parts, self._u64(mult)


def _sharded_query(seed):
    from paper_2206_10435_gb300 import datagen as G
    # a chain and a star-shaped tree (a relation with two children); seed 0:
    # two rows per relation, so a third rank holds no rows at all
    if seed == 0:
        return G.chain3_uniform(seed=11, rows=2, end_domain=2, mid_domain=1)
    if seed % 2:
        return G.chain3_uniform(seed=seed, rows=400, end_domain=60, mid_domain=12)
    q = G.chain3_uniform(seed=seed, rows=300, end_domain=40, mid_domain=10)
    R = q.relations
    extra = G.Relation("R4", [R[0].attrs[1], 99], [R[1].keys[0][::-1].copy(), R[2].keys[1].copy()], [])
    return G.Query("tree", R + [extra], q.attr_names)


def _rank_sharded(rank, world, port, out, seed):
    dist = _init(rank, world, port)
    from paper_2206_10435_gb300 import shard as S
    q = _sharded_query(seed)
    eng = NumpyShard(q, rank, world)
    total, up, down, mult = S.sharded_summary(dist, eng, eng.parent)
    local = {t: [(tuple(int(x) for x in k), int(m)) for k, m in zip(eng.local_keys[t], mult[t])]
             for t in mult}
    out.put((rank, total, local))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,seed", [(2, 3), (2, 4), (3, 3), (3, 4), (3, 0)])
def test_gloo_ranks_row_sharded_counting_matches_the_oracle(world, seed):
    """Every relation split by rows over two or three ranks (rows not a
    multiple of the rank count; with seed 0 one rank holds no rows): the total
    and every key tuple's multiplicity (summed over the ranks' local groups)
    equal the oracle's counting pass on the whole relations."""
    from oracle import oracle as O
    res = _spawn(_rank_sharded, world, seed)
    q = _sharded_query(seed)
    c = O.count(q, rows=True)
    assert len(res) == world
    assert all(r[1] == int(c.total) for r in res) and int(c.total) > 0
    want = O.group_mult_from_counts(q, c)
    for t, (allk, m) in enumerate(want):
        got = {}
        for _, _, local in res:
            for k, v in local[t]:
                got[k] = got.get(k, 0) + v
        ref = {tuple(int(x) for x in k): int(v) for k, v in zip(allk, m)}
        assert {k: v for k, v in got.items() if v} == {k: v for k, v in ref.items() if v}, t
