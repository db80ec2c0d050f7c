"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the barrier,
the max-over-ranks time and the whole-job throughput of replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (world, rank, rank)
    bench.barrier()
    my_seconds = 1.0 + rank          # rank 1 is the slow one
    m = bench.reduce_max(my_seconds)
    out[rank] = (m, bench.aggregate_throughput(10_000, world, m))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        m, value = out[r]
        assert m == pytest.approx(2.0)                   # max over ranks
        assert value == pytest.approx(2 * 10_000 / 2.0)  # all ranks' queries / slowest time


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.aggregate_throughput(100, 1, 0.5) == 200
