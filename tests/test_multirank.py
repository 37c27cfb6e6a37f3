"""The benchmark's multi-GPU reduction (slowest rank's time, rows of all
ranks) run as world_size-2 gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 100 + 50 r ms and produced 1000 (r + 1) rows
    t, rows = bench.reduce_over_ranks(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
    dist.barrier()
    out.put((rank, t, rows))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_rows():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 150.0, 3000), (1, 150.0, 3000)]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7, "cpu") == (12.5, 7)
