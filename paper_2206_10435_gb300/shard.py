"""The counting pass of a row-sharded query across ranks.

Every relation is split by rows across the ranks (``rows_of`` gives rank r
its contiguous share); each rank loads its rows and creates the query as
usual.  The pass then follows the join tree edge by edge (Algorithm 2,
Section 3.3): leaves to root, each rank computes its partial message to the
parent from its own rows and the children's global messages, and one exact
saturating sum over the ranks (``partition.sum_sat``) makes the global
message; the root's partial sums give |Q|.  Root to leaves, the down
messages go the same way.  The result: |Q|, every edge's global up and down
messages, and each rank's partial multiplicities of its local groups (the
ranks' values for one key tuple add up to that key tuple's marginal over
the result, Section 1.2).

The per-rank work is an ``engine`` with the calls of ``GpuShard`` (the C
ABI's gj_shard_*); messages travel as uint64 numpy vectors over the
separator attribute's value domain, which the ranks agree on first.
"""
from __future__ import annotations

import numpy as np

from . import partition as P


def rows_of(n_rows: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of a relation of n_rows rows that rank `rank` holds."""
    return P.row_range(n_rows, rank, world)


def preorder(parent) -> list:
    """Positions of the join tree in preorder from the root (position 0),
    children in position order."""
    children = {j: [] for j in range(len(parent))}
    for j, p in enumerate(parent):
        if p >= 0:
            children[p].append(j)
    out, stack = [], [0]
    while stack:
        t = stack.pop()
        out.append(t)
        stack.extend(reversed(children[t]))
    return out


def agree_domains(dist, local: dict, device="cpu") -> dict:
    """{rel: (lo, length)} of every separator domain: the union over ranks of
    the local ranges {rel: (lo, hi)}."""
    rels = sorted(local)
    lo = np.array([local[r][0] for r in rels], dtype=np.int64)
    hi = np.array([local[r][1] for r in rels], dtype=np.int64)
    if dist is not None and rels:
        import torch
        tl = torch.from_numpy(lo).to(device)
        th = torch.from_numpy(hi).to(device)
        dist.all_reduce(tl, op=dist.ReduceOp.MIN)
        dist.all_reduce(th, op=dist.ReduceOp.MAX)
        lo, hi = tl.cpu().numpy(), th.cpu().numpy()
    out = {}
    for r, a, b in zip(rels, lo.tolist(), hi.tolist()):
        out[r] = (int(a), int(b - a + 1)) if a <= b else (0, 1)   # no rows anywhere: one empty slot
    return out


def sharded_summary(dist, engine, parent, device="cpu"):
    """The row-sharded counting pass.  Returns (|Q| (2^64 - 1 means 2^64 - 1
    or more), up messages {rel: (vector, lo)}, down messages {rel: (vector,
    lo)}, this rank's partial multiplicities {rel: vector over its local
    groups})."""
    pre = preorder(parent)
    children = {t: [j for j, p in enumerate(parent) if p == t] for t in range(len(parent))}
    dom = agree_domains(dist, {t: engine.shard_domain(t) for t in pre if parent[t] >= 0}, device)
    up, total = {}, None
    for t in reversed(pre):
        msgs = {c: up[c] for c in children[t]}
        lo, length = dom.get(t, (0, 1))
        part = engine.shard_up(t, msgs, lo, length)
        glob = P.sum_sat(dist, part, device)
        if parent[t] < 0:
            total = int(glob[0])
        else:
            up[t] = (glob, lo)
    down, mult = {}, {}
    for t in pre:
        parts, mult[t] = engine.shard_down(t, down.get(t), {c: up[c] for c in children[t]})
        for c, part in parts.items():
            down[c] = (P.sum_sat(dist, part, device), up[c][1])
    return total, up, down, mult


class GpuShard:
    """One rank's engine on its GPU: a gj.Query over the rank's rows."""

    def __init__(self, query):
        self.q = query
        self.torch = query.ctx.torch
        self.dev = self.torch.device("cuda", query.ctx.device)
        # messages move on the context's stream, in order with its kernels
        self.stream = query.ctx.stream

    def _dev(self, msgs):
        return {c: (self.torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).to(self.dev), lo)
                for c, (v, lo) in msgs.items()}

    @staticmethod
    def _host(t):
        return t.cpu().numpy().view(np.uint64).copy()

    def shard_domain(self, rel):
        return self.q.shard_domain(rel)

    def shard_up(self, rel, msgs, lo, length):
        with self.torch.cuda.stream(self.stream):
            return self._host(self.q.shard_up(rel, self._dev(msgs), lo, length))

    def shard_down(self, rel, down, msgs):
        with self.torch.cuda.stream(self.stream):
            d = self._dev({rel: down})[rel] if down is not None else None
            parts, mult = self.q.shard_down(rel, d, self._dev(msgs))
            return {c: self._host(v) for c, v in parts.items()}, self._host(mult)
