"""Sharding of the batched workload's independent instances over ranks, on
the CPU: every instance is owned by exactly one rank and the load is balanced;
two gloo ranks that each run their shard (the oracle stands in for the
device here) and sum their counters get the single-process totals."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

from paper_2509_26361_gb300 import sharding
from paper_2509_26361_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_instance_is_owned_once_and_the_load_is_balanced():
    cells = [n ** 3 for n in W.batched_sizes()]
    assert len(cells) == 64
    for world in (1, 2, 3, 4, 8):
        parts = sharding.shard(cells, world)
        owned = sorted(i for p in parts for i in p)
        assert owned == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        # greedy largest-first: every rank within one instance of the mean
        assert max(loads) - sum(loads) / world <= max(cells)
        assert parts == sharding.shard(cells, world)  # deterministic
        assert all(sharding.owned_by(cells, r, world) == parts[r] for r in range(world))


def _instances():
    """Eight small independent instances (sizes 12-20, own fields and spheres)."""
    rng = np.random.default_rng(41)
    out = []
    for n in (16, 12, 20, 16, 12, 20, 16, 12):
        sp = W.random_spheres(rng, 1, 2.6 / n, 0.3, n)
        phi, faces = W.sphere_phi_nodes_faces((n, n, n), sp)
        out.append((n, phi, faces, W.fourier_velocity((n, n, n), rng)))
    return out


def _counters(insts, which):
    """Event counters (markers, annihilations, multi, inconsistent, CFL) of two
    steps of the given instances, summed."""
    import oracle

    tot = np.zeros(5)
    for i in which:
        n, phi, faces, u = insts[i]
        st = oracle.init(phi, faces)
        for k in range(2):
            for d in ((0, 1, 2) if k % 2 == 0 else (2, 1, 0)):
                st, c = oracle.sweep(st, d, u[d], 0.5)
                tot += c
    return tot


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
    insts = _instances()
    mine = sharding.owned_by([n ** 3 for n, *_ in insts], rank, world)
    out[rank] = (mine, bench.sum_over_ranks(list(_counters(insts, mine)), world, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_batch_once():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out[0][0] + out[1][0]) == list(range(8))
    assert not set(out[0][0]) & set(out[1][0])
    ref = _counters(_instances(), range(8))
    assert ref[0] > 0
    assert out[0][1] == out[1][1] == list(ref)
