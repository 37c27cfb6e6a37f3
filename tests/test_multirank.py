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
