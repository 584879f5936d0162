"""The z-slab decomposition of one grid (paper_2509_26361_gb300/slab.py) on the
CPU: ranks that each step their slab, refreshing two halo layers after every
split sweep, end in exactly the single-domain state, and Front2VOF on each
rank's owned cells gives the single-domain fractions.  The oracle is the
per-rank engine here; on a GPU node it is the CUDA library (GridEngine)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2509_26361_gb300 import slab as S
from paper_2509_26361_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N3 = (24, 20, 40)
STEPS = 2


def _problem():
    """Lumpy shapes (thin features, saddle faces) in a divergence-free field."""
    rng = np.random.default_rng(17)
    sp = [W.Sphere(tuple(rng.uniform(0, 1, 3)), rng.uniform(0.08, 0.2)) for _ in range(7)]
    phi, faces = W.sphere_phi_nodes_faces(N3, sp)
    u = W.fourier_velocity(N3, rng)
    lams = [0.8 if k % 2 == 0 else -0.6 for k in range(STEPS)]
    return phi, faces, u, lams


def _oracle_engine(cb, s, d, u_d, lam):
    st, _ = oracle.sweep(oracle.State(cb.numpy(), s.numpy()), d, u_d, lam)
    return torch.from_numpy(np.ascontiguousarray(st.cb)), torch.from_numpy(np.ascontiguousarray(st.s))


def _reference():
    phi, faces, u, lams = _problem()
    st = oracle.init(phi, faces)
    for n, lam in enumerate(lams):
        st = oracle.step(st, n, u, lam)
    C, _ = oracle.front2vof(st)
    return st.cb, st.s, C


def _run_rank(rank, world):
    phi, faces, u, lams = _problem()
    st0 = oracle.init(phi, faces)
    sl = S.Slab(N3[2], rank, world)
    cb = torch.from_numpy(sl.cut(st0.cb))
    s = torch.from_numpy(sl.cut(st0.s))
    ul = [sl.cut(u[d]) for d in range(3)]
    cb, s = S.run_steps(sl, _oracle_engine, cb, s, ul, lams)
    C, _ = oracle.front2vof(oracle.State(cb.numpy(), s.numpy()))
    return sl, sl.owned(cb.numpy()), sl.owned(s.numpy()), sl.owned(C)


def _free_port():
    so = socket.socket()
    so.bind(("127.0.0.1", 0))
    port = so.getsockname()[1]
    so.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sl, cb, s, C = _run_rank(rank, world)
    out[rank] = (sl.z0, sl.z1, cb, s, C)
    dist.barrier()
    dist.destroy_process_group()


def test_owned_ranges_cover_the_grid_once():
    for nz in (16, 40, 41):
        for world in (1, 2, 3, 5):
            r = [S.owned_range(nz, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == nz
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


def test_one_rank_slab_equals_the_global_run():
    cb_r, s_r, C_r = _reference()
    sl, cb, s, C = _run_rank(0, 1)
    assert np.array_equal(cb, cb_r)
    assert np.array_equal(s.view(np.uint64), s_r.view(np.uint64))
    assert np.array_equal(C, C_r)


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_with_halo_exchange_equal_the_global_run(world):
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    cb_r, s_r, C_r = _reference()
    c = cb_r & 1
    changed = 0
    for k in range(world):
        z0, z1, cb, s, C = out[k]
        assert np.array_equal(cb, cb_r[z0:z1]), f"rank {k}: colours differ"
        assert np.array_equal(s.view(np.uint64), s_r[:, z0:z1].view(np.uint64)), f"rank {k}: offsets differ"
        assert np.array_equal(C, C_r[z0:z1]), f"rank {k}: fractions differ"
        changed += int(np.sum(c[z0:z1] != np.roll(c, -1, axis=0)[z0:z1]))
    assert changed > 0  # markers cross the slab boundaries


def _emulated_errors(halo):
    """Sweeps after which a rank's owned layers differ from the global run,
    with the halos reloaded from the global state after every sweep (the
    exchange, emulated in one process), for two ranks."""
    phi, faces, u, lams = _problem()
    st0 = oracle.init(phi, faces)
    bad = 0
    for rank in range(2):
        sl = S.Slab(N3[2], rank, 2, halo=halo)
        cb, s = torch.from_numpy(sl.cut(st0.cb)), torch.from_numpy(sl.cut(st0.s))
        ul = [sl.cut(u[d]) for d in range(3)]
        stg = st0
        for n, lam in enumerate(lams):
            for d in ((0, 1, 2) if n % 2 == 0 else (2, 1, 0)):
                cb, s = _oracle_engine(cb, s, d, ul[d], lam)
                stg, _ = oracle.sweep(stg, d, u[d], lam)
                same = (np.array_equal(sl.owned(cb.numpy()), stg.cb[sl.z0:sl.z1]) and
                        np.array_equal(sl.owned(s.numpy()), stg.s[:, sl.z0:sl.z1]))
                bad += not same
                cb, s = torch.from_numpy(sl.cut(stg.cb)), torch.from_numpy(sl.cut(stg.s))
    return bad


def test_two_halo_layers_are_needed():
    """The halo depth follows the sweep's reach along z: the circle fits of a
    z sweep use polyline neighbours two cells away, so one layer leaves wrong
    offsets next to the slab boundaries and two layers do not."""
    assert _emulated_errors(1) > 0
    assert _emulated_errors(2) == 0
