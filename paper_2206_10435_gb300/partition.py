"""Work partitions across ranks (one process per GPU) and the collectives
that join their results.

Two partitions of the hot path need no exchange of data between ranks:

* one large query: every rank builds the same factors and summary (the
  summary is O(input), the result O(|Q|)), then desummarises its own
  contiguous range of the result rows.  Ranges are equal to within one row,
  so the work of the dominant step is split evenly; concatenated in rank
  order they are the whole result in canonical order.
* many independent queries (batched or served): rank r takes a contiguous
  block of the query list; per-query results are gathered back in query
  order.

The counting pass of a row-sharded query (every relation split by rows
across ranks) needs one exact saturating sum per tree edge: ``sum_sat``
adds uint64 vectors across ranks exactly, saturating at 2^64 - 1 like the
semiring of the summary.

``dist`` is ``torch.distributed`` (NCCL on GPUs, gloo on the CPU) or None
for a single process.
"""
from __future__ import annotations

import numpy as np

SAT = (1 << 64) - 1


def row_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of a result of `total` rows that rank `rank` of `world`
    desummarises: equal contiguous shares, the first total % world ranks
    one row more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    q, r = divmod(int(total), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def windows(lo: int, hi: int, chunk: int):
    """(row0, n) windows of at most `chunk` rows covering [lo, hi)."""
    if chunk < 1:
        raise ValueError("chunk must be positive")
    return [(r0, min(chunk, hi - r0)) for r0 in range(lo, hi, chunk)]


def query_block(n_queries: int, rank: int, world: int) -> tuple[int, int]:
    """Queries [lo, hi) of a list of n_queries that rank `rank` handles."""
    return row_range(n_queries, rank, world)


def _as_tensor(torch, values, device, dtype):
    return torch.as_tensor(np.asarray(values), dtype=dtype).to(device)


def max_over_ranks(dist, x: float, device="cpu") -> float:
    """The largest x over ranks (the slowest rank's time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_in_order(dist, local: np.ndarray, n_total: int, rank: int, world: int,
                    device="cpu") -> np.ndarray:
    """Per-query uint64 results of every rank, concatenated in query order:
    rank r holds the block query_block(n_total, r, world).  Every rank gets
    the whole vector."""
    local = np.ascontiguousarray(local, dtype=np.uint64)
    lo, hi = query_block(n_total, rank, world)
    if local.shape[0] != hi - lo:
        raise ValueError("local results do not match the rank's query block")
    if dist is None:
        return local.copy()
    import torch
    # the all-gather moves equal-sized pieces: pad every block to the largest
    size = -(-n_total // world)
    piece = np.zeros(size, dtype=np.uint64)
    piece[:local.shape[0]] = local
    t = _as_tensor(torch, piece.view(np.int64), device, torch.int64)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out = np.empty(n_total, dtype=np.uint64)
    for r in range(world):
        a, b = query_block(n_total, r, world)
        out[a:b] = parts[r].cpu().numpy().view(np.uint64)[:b - a]
    return out


def sum_sat(dist, values: np.ndarray, device="cpu") -> np.ndarray:
    """Element-wise sum over ranks of uint64 vectors, exact, saturating at
    2^64 - 1 (SAT; a SAT input stays SAT).  Each value is split into its
    32-bit halves; the halves are summed as int64 (exact below 2^31 ranks)
    and the saturation marks reduced by max, then the 128-bit sums are put
    back together."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    if dist is None:
        return v.copy()
    import torch
    lo = (v & np.uint64(0xFFFFFFFF)).astype(np.int64)
    hi = (v >> np.uint64(32)).astype(np.int64)
    sat = (v == np.uint64(SAT)).astype(np.int64)
    lo[sat == 1] = 0
    hi[sat == 1] = 0
    t = _as_tensor(torch, np.stack([lo, hi]), device, torch.int64)
    s = _as_tensor(torch, sat, device, torch.int64)
    dist.all_reduce(t)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    lo_s, hi_s = t.cpu().numpy()
    sat_s = s.cpu().numpy() != 0
    # value = hi_s * 2^32 + lo_s; it reaches 2^64 - 1 iff the carry into the
    # top half leaves 32 bits, or the value is exactly SAT
    top = hi_s + (lo_s >> 32)
    sat_s |= top >= (1 << 32)
    val = ((top.astype(np.uint64) & np.uint64(0xFFFFFFFF)) << np.uint64(32)) | \
        (lo_s.astype(np.uint64) & np.uint64(0xFFFFFFFF))
    sat_s |= val == np.uint64(SAT)
    val[sat_s] = np.uint64(SAT)
    return val
