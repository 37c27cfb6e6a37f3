"""The row-sharded counting pass with the GPU engine (gj_shard_* through
the C ABI): two or three ranks, each a host thread with its own context and
stream on the one GPU, holding its rows of every relation.  Their partial
messages are exchanged on the host through a group of the threads (the
collectives of torch.distributed that the coordinator calls, done between
the threads); no kernel waits on another.  One case gives a rank no rows at
all.  The total and every key tuple's multiplicity must equal the oracle's,
and with one rank they equal gj_summarize's."""
import threading

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_10435_gb300 import datagen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class _ThreadGroup:
    """all_reduce between the threads of one process (SUM, MIN, MAX)."""

    class ReduceOp:
        SUM, MIN, MAX = "sum", "min", "max"

    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.slots = [None] * world

    def member(self, rank):
        g = self

        class _M:
            ReduceOp = _ThreadGroup.ReduceOp

            def all_reduce(self, t, op="sum"):
                g.slots[rank] = t.clone()
                g.barrier.wait()
                vals = [g.slots[r] for r in range(g.world)]
                if op == "sum":
                    r = sum(vals[1:], vals[0].clone())
                elif op == "min":
                    r = torch.stack(vals).min(dim=0).values
                else:
                    r = torch.stack(vals).max(dim=0).values
                g.barrier.wait()
                t.copy_(r)
        return _M()


def _shard_query(seed):
    if seed == 1:   # two rows per relation: a third rank holds none
        return G.chain3_uniform(seed=11, rows=2, end_domain=2, mid_domain=1)
    if seed == 0:
        return G.chain_query("c4", [2000, 3000, 1500, 2500], [300, 40, 60, 50, 200], [1.0] * 5,
                             np.int64, seed=G.SEED_BASE + 70)
    q = G.chain3_uniform(seed=seed, rows=4000, end_domain=500, mid_domain=50)
    R = q.relations
    extra = G.Relation("R4", [R[0].attrs[1], 99], [R[1].keys[0][::-1].copy(), R[2].keys[1].copy()], [])
    return G.Query("tree", R + [extra], q.attr_names)


def _run_rank(q, rank, world, group, out):
    from paper_2206_10435_gb300 import gj, shard as S
    try:
        ctx = gj.Context(0, torch.cuda.Stream())
        ids = []
        for R in q.relations:
            lo, hi = S.rows_of(R.n_rows, rank, world)
            keys = [torch.from_numpy(np.ascontiguousarray(k[lo:hi])).cuda() for k in R.keys]
            torch.cuda.synchronize()
            ids.append(ctx.load_relation(keys, R.attrs))
        qq = ctx.query(ids)
        eng = S.GpuShard(qq)
        total, up, down, mult = S.sharded_summary(group.member(rank) if group else None, eng, qq.parent)
        local = {}
        for t in range(len(q.relations)):
            R = q.relations[t]
            lo, hi = S.rows_of(R.n_rows, rank, world)
            sep = [c for c, a in enumerate(R.attrs) if t and a in _seen_before(q, t)]
            order = sep + [c for c in range(len(R.attrs)) if c not in sep]
            _, _, gkey = ctx.factor_export(ids[t], hi - lo, len(R.keys), order)
            keys = gkey.cpu().numpy().T
            local[t] = [(tuple(int(x) for x in k), int(m)) for k, m in zip(keys, mult[t])]
        qq.close()
        for i in ids:
            ctx.release_relation(i)
        ctx.close()
        out[rank] = (total, local)
    except BaseException as e:   # surfaced by the test
        out[rank] = e


def _seen_before(q, t):
    return {a for R in q.relations[:t] for a in R.attrs}


@pytest.mark.parametrize("world,seed", [(2, 0), (2, 5), (3, 5), (3, 1)])
def test_row_sharded_counting_on_several_ranks_matches_the_oracle(world, seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q = _shard_query(seed)
    group = _ThreadGroup(world)
    out = [None] * world
    th = [threading.Thread(target=_run_rank, args=(q, r, world, group, out)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    for r in out:
        if isinstance(r, BaseException):
            raise r
    c = O.count(q, rows=True)
    assert all(r[0] == int(c.total) for r in out) and int(c.total) > 0
    for t, (allk, m) in enumerate(O.group_mult_from_counts(q, c)):
        got = {}
        for _, local in out:
            for k, v in local[t]:
                got[k] = got.get(k, 0) + v
        ref = {tuple(int(x) for x in k): int(v) for k, v in zip(allk, m)}
        assert {k: v for k, v in got.items() if v} == {k: v for k, v in ref.items() if v}, t


def test_one_rank_equals_the_summary():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj, shard as S
    from tests.gpu_util import Run, to_u64
    q = _shard_query(5)
    ctx = gj.Context(0)
    run = Run(ctx, q)
    total = run.summarize()
    t_sh, up, down, mult = S.sharded_summary(None, S.GpuShard(run.q), run.q.parent)
    assert t_sh == total
    for t in range(len(q.relations)):
        _, m, _ = run.q.summary_groups(t)
        assert np.array_equal(mult[t], to_u64(m))
    run.close()
    ctx.close()
