"""The multi-GPU path of the bench is replicas only (independent instances, no data-path
collective): each rank times its own steps and the job takes the slowest rank.  This covers that
host logic with world_size 2 on CPU (gloo)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 200.0][rank]   # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist, "cpu")
    sps, value = bench.replica_rate(10, m, world)
    q.put((rank, m, sps, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, sps, value in out:
        assert m == 200.0
        assert sps == pytest.approx(50.0) and value == pytest.approx(100.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(123.0) == 123.0
    assert bench.replica_rate(5, 1000.0, 1) == (5.0, 5.0)
