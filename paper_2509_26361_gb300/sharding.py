"""Sharding of independent EBIT instances over ranks (one process per GPU).

The batched workload (many instances of different grid sizes, each with its
own velocity field) has no data dependence between instances, so a job on N
GPUs gives every rank a disjoint subset and runs it as its own batch: no
collective on the data path, only a reduction of the timings and counters at
the end.  The partition is deterministic (every rank computes the same one
from the instance sizes alone) and balanced by cell count: instances in
decreasing size, each to the rank with the fewest cells so far (ties to the
lower rank), which leaves every rank within one instance of the mean load.

A single large grid does not shard this way: a split sweep needs the state of
neighbouring planes (one layer of halo across the sweep for the x and y
sweeps, two along z for the z sweep, one for Front2VOF and five for the
height-function columns), so its partition is a slab decomposition with a halo
exchange per sweep; this library runs one grid per GPU.
"""
from __future__ import annotations


def shard(cells, world):
    """Owner rank of each instance: ``cells[i]`` is the cell count of instance
    i.  Returns a list of ``world`` lists of instance indices (each in
    increasing order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-cells[i], i))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(i)
        load[r] += cells[i]
    return [sorted(o) for o in owned]


def owned_by(cells, rank, world):
    """The instances of ``rank`` (see shard)."""
    return shard(cells, world)[rank]
