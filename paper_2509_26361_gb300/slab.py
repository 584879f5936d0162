"""Slab decomposition of one grid over ranks along z, with a halo exchange
after every split sweep.

The paper runs its weak-scaling tests with a Cartesian domain decomposition
(Sec. 3.1, Table 1).  Here a grid of nx x ny x nz nodes is split into
contiguous z-slabs, one per rank.  Each rank keeps its slab plus HALO node
layers on each side (periodic in z across the ranks) and treats that local
grid as its own periodic domain.  A split sweep changes a node only from the
state within two layers of it:
- the band pass reads its colour window from one layer behind to two ahead;
- the FP64 lists read the plane window of an unaligned edge from one layer
  behind to two ahead across the sweep, and two on each side along it.

So with HALO = 2 every owned layer is exact after a sweep, while the halos,
fed from the far side of the local grid's wrap, are not.  The exchange then
overwrites each rank's halos with the neighbours' owned layers before the next
sweep.  Front2VOF of an owned cell reads one node layer ahead, which the
refreshed halo holds.

The exchange is point to point over torch.distributed: NCCL between GPUs,
gloo on the CPU.  It sends the colour bytes and the three offset planes, in
two phases (upward, then downward) so that two ranks that are each other's
only neighbour still match sends to receives.  The per-rank engine is anything
that advances a local state by one sweep: the CUDA library (GridEngine) on a
GPU node, or the CPU oracle in the tests.
"""
from __future__ import annotations

import numpy as np
import torch

HALO = 2


def owned_range(nz, rank, world):
    """The z-layers [z0, z1) that ``rank`` owns (contiguous, sizes differing by
    at most one)."""
    return rank * nz // world, (rank + 1) * nz // world


class Slab:
    """One rank's slab: owned layers [z0, z1) and HALO layers on each side."""

    def __init__(self, nz, rank, world, halo=HALO):
        self.nz, self.rank, self.world, self.halo = nz, rank, world, halo
        self.z0, self.z1 = owned_range(nz, rank, world)
        if self.z1 - self.z0 < halo:
            raise ValueError("every rank needs at least HALO owned layers")

    @property
    def nz_local(self):
        return self.z1 - self.z0 + 2 * self.halo

    def cut(self, arr):
        """The local copy (owned layers and halos, periodic in z) of a global
        array whose third axis from the end is z."""
        zs = np.arange(self.z0 - self.halo, self.z1 + self.halo) % self.nz
        return np.ascontiguousarray(np.take(np.asarray(arr), zs, axis=-3))

    def owned(self, local):
        """The owned layers of a local array."""
        h = self.halo
        return local[..., h:local.shape[-3] - h, :, :]

    def exchange(self, local):
        """Refresh the halos of a local torch tensor (z third from the end) in
        place from the neighbouring ranks' owned layers."""
        import torch.distributed as dist

        h = self.halo
        nzl = local.shape[-3]
        top_owned = local[..., nzl - 2 * h:nzl - h, :, :].contiguous()
        bottom_owned = local[..., h:2 * h, :, :].contiguous()
        if self.world == 1:
            local[..., 0:h, :, :] = top_owned
            local[..., nzl - h:nzl, :, :] = bottom_owned
            return local
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        recv_bottom = torch.empty_like(top_owned)
        recv_top = torch.empty_like(bottom_owned)
        # upward: my top owned layers become the upper neighbour's bottom halo
        ops = [dist.P2POp(dist.isend, top_owned, up), dist.P2POp(dist.irecv, recv_bottom, down)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        # downward: my bottom owned layers become the lower neighbour's top halo
        ops = [dist.P2POp(dist.isend, bottom_owned, down), dist.P2POp(dist.irecv, recv_top, up)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        local[..., 0:h, :, :] = recv_bottom
        local[..., nzl - h:nzl, :, :] = recv_top
        return local


def run_steps(slab, engine, cb, s, u, lams, first_step=0):
    """Advance a local state (colour bytes cb [nz_l, ny, nx], offsets s
    [3, nz_l, ny, nx], torch tensors) by len(lams) steps of three split sweeps
    (x-y-z on even steps, z-y-x on odd), refreshing the halos after every sweep.
    ``engine(cb, s, d, u_d, lam)`` returns the swept local state; ``u`` holds
    the three local velocity fields."""
    for k, lam in enumerate(lams):
        n = first_step + k
        for d in ((0, 1, 2) if n % 2 == 0 else (2, 1, 0)):
            cb, s = engine(cb, s, d, u[d], lam)
            slab.exchange(cb)
            slab.exchange(s)
    return cb, s


class GridEngine:
    """The CUDA library as a slab engine: a context over the local grid.  Each
    sweep loads the exchanged state (ebit_set_state), so the context's first
    sweep after it processes every tile; the state is read back for the next
    exchange."""

    def __init__(self, n3_local, h):
        from . import ebit

        self.g = ebit.Grid(*n3_local, h=h)

    def __call__(self, cb, s, d, u_d, lam):
        self.g.set_state(cb, s)
        self.g.sweep(d, u_d, lam * self.g.h)
        return self.g.get_state()

    def close(self):
        self.g.close()
