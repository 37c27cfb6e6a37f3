"""Helpers for the GPU parity tests: run a datagen.Query through the C ABI
(libgj.so) and bring results back as numpy arrays."""
import numpy as np

from oracle import oracle as O


def to_u64(t):
    """int64 torch tensor holding uint64 bit patterns -> numpy uint64."""
    return t.cpu().numpy().view(np.uint64)


class Run:
    def __init__(self, ctx, query, drop=()):
        from paper_2206_10435_gb300 import gj
        self.ctx = ctx
        self.query = query
        self.ids = gj.load_query(ctx, query)
        self.q = ctx.query(self.ids, drop_attrs=drop)
        self.plan = O.plan(query, drop)

    def summarize(self):
        return self.q.summarize()

    def rows(self, row0=0, n=None):
        """Result rows [row0, row0+n): (columns, row ids [n, k])."""
        if n is None:
            n = self.q.total - row0
        cols, rids = self.q.desummarize(row0, n, rowids=True)
        return ([c.cpu().numpy() for c in cols],
                np.stack([r.cpu().numpy() for r in rids], axis=1))

    def factor_order(self, rel):
        """Column order of the relation's factor in this query: separator
        columns (declared order), then the others."""
        R = self.query.relations[rel]
        sep = [c for c, a in enumerate(R.attrs) if a in self.plan.sep[rel]]
        return sep + [c for c in range(len(R.attrs)) if c not in sep]

    def group_table(self, rel):
        """{key tuple (declared column order): (w, mult)} of a relation."""
        R = self.query.relations[rel]
        perm, gstart, gkey = self.ctx.factor_export(self.ids[rel], R.n_rows, len(R.keys),
                                                    self.factor_order(rel))
        w, m, o = self.q.summary_groups(rel)
        keys = gkey.cpu().numpy().T
        return {tuple(k): (int(a), int(b)) for k, a, b in
                zip(keys.tolist(), to_u64(w).tolist(), to_u64(m).tolist())}

    def close(self):
        self.q.close()
        for i in self.ids:
            self.ctx.release_relation(i)


def device_columns(torch, query, device="cuda"):
    """Device copies of every relation's key and payload columns."""
    keys = [[torch.from_numpy(k).to(device) for k in R.keys] for R in query.relations]
    pays = [[torch.from_numpy(p).to(device) for p in R.payloads] for R in query.relations]
    return keys, pays


def check_canonical_window(torch, query, plan, dev, cols, rids, prev_last=None):
    """Properties that make a window of rows exactly a slice of the sorted
    join result: every row is a join tuple (each relation's keys at its row
    id equal the row's V values), payloads are those of the row ids, and rows
    strictly increase in canonical order (V values, then row ids).  Works on
    device tensors of any size.  Returns the window's last row key."""
    nv = len(plan.V)
    for j, R in enumerate(query.relations):
        rj = rids[j].long()
        for c, a in enumerate(R.attrs):
            src = dev[0][j][c]
            assert torch.equal(src[rj], cols[plan.V.index(a)]), (j, c)
    pc = nv
    for j, R in enumerate(query.relations):
        rj = rids[j].long()
        for p in range(len(R.payloads)):
            assert torch.equal(dev[1][j][p][rj], cols[pc]), (j, p)
            pc += 1
    keycols = [cols[v].long() for v in range(nv)] + [r.long() for r in rids]
    n = keycols[0].shape[0]
    if n > 1:
        less = torch.zeros(n - 1, dtype=torch.bool, device=keycols[0].device)
        eq = torch.ones(n - 1, dtype=torch.bool, device=keycols[0].device)
        for x in keycols:
            less |= eq & (x[:-1] < x[1:])
            eq &= x[:-1] == x[1:]
        assert bool(less.all()), "rows not strictly increasing in canonical order"
    first = [int(x[0]) for x in keycols]
    if prev_last is not None:
        assert tuple(prev_last) < tuple(first), "window boundary out of order"
    return [int(x[-1]) for x in keycols]
