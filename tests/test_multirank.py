"""Multi-process host logic of bench.py on CPU ranks (gloo, world size 2):
every rank times its own independent system; the job reports the units of
all ranks over the slowest rank's time (max over ranks), with no data-path
collective."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    local = [1.0 + rank, 2.0 - rank]           # rank 1 is slower on the first timer
    got = bench.reduce_max(local, dist, device="cpu")
    value, tmax = bench.aggregate([got[0]], [512 * 2 * world])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, value, tmax))


def test_max_over_ranks_and_whole_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value, tmax in res:
        assert got == [2.0, 2.0]               # max over ranks, element-wise
        assert tmax == 2.0
        assert value == pytest.approx(512 * 2 * world / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.aggregate([2.0], [1024]) == (512.0, 2.0)
