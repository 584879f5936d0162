"""Multi-rank logic of bench.py on the CPU: two gloo ranks (replicas of the
workload, one per GPU on a GPU node) agree on the slowest rank's time and the
whole-job value counts every rank's cells."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 25.0 * rank          # rank 1 is the slower one
    m = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (m, bench.job_value(128 ** 3, 512, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 125.0
    assert out[0][1] == pytest.approx(128 ** 3 * 512 * 2 / 0.125)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.job_value(10, 3, 1, 1000.0) == 30.0
