"""Batched persistent sweeps (one cooperative launch per split sweep for all
instances, CUDA-graph replay of whole steps): every instance must end in the
state a separate context reaches from the same inputs (colour bytes and
offsets bit for bit, the same event counters), and a small instance must
match the CPU FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def instances(seed, sizes):
    """Each instance: its own seeded 12-mode Fourier field and 1-3 spheres."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        k = int(rng.integers(1, 4)) if n >= 16 else 1
        rmin = 2.5 / n
        sp = W.random_spheres(rng, k, rmin, max(0.16, rmin + 0.05), n)
        phi, faces = W.sphere_phi_nodes_faces((n, n, n), sp)
        u = W.fourier_velocity((n, n, n), rng)
        out.append((n, phi, faces, u))
    return out


def make_batch(insts, cfl=0.5):
    b = ebit.Batch([(n, n, n) for n, *_ in insts])
    uf = []
    for i, (n, phi, faces, u) in enumerate(insts):
        b.instance(i).init(dev(phi), dev(faces))
        uf.append(tuple(dev(u[d]) for d in range(3)))
    b.set_velocity(uf, [cfl / n for n, *_ in insts])
    return b


def reference_states(insts, steps, cfl=0.5):
    out = []
    for n, phi, faces, u in insts:
        g = ebit.Grid(n, n, n)
        g.init(dev(phi), dev(faces))
        ud = [dev(u[d]) for d in range(3)]
        for k in range(steps):
            g.step(k, ud, cfl / n)
        cb, s = g.get_state()
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.front2vof(C)
        out.append((cb.cpu(), s.cpu(), C.cpu(), g.counters()))
        g.close()
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_separate_contexts(graph):
    insts = instances(4, [16, 24, 32, 16, 40, 24, 8])
    steps = 7
    ref = reference_states(insts, steps)
    b = make_batch(insts)
    b.run(0, steps, graph=graph)
    b.sync()
    for i, (cb_r, s_r, C_r, cnt_r) in enumerate(ref):
        g = b.instance(i)
        cb, s = g.get_state()
        assert torch.equal(cb.cpu(), cb_r), f"instance {i}: colours differ"
        assert torch.equal(s.cpu(), s_r), f"instance {i}: offsets differ"
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.front2vof(C)
        assert torch.equal(C.cpu(), C_r), f"instance {i}: volume fractions differ"
        assert g.counters() == cnt_r, (i, g.counters(), cnt_r)
    if graph:
        assert b.graph_active() in (1, 2), b.graph_note()
    b.close()


def test_batch_instance_matches_oracle():
    insts = instances(9, [16, 24])
    b = make_batch(insts)
    osts = [oracle.init(phi, faces) for _, phi, faces, _ in insts]
    for k in range(3):
        order = (0, 1, 2) if k % 2 == 0 else (2, 1, 0)
        for d in order:
            b.sweep(d)
            osts = [oracle.sweep(o, d, u[d], 0.5)[0] for o, (_, _, _, u) in zip(osts, insts)]
    b.sync()
    for i, o in enumerate(osts):
        cb, s = b.instance(i).get_state()
        cb, s = cb.cpu().numpy(), s.cpu().numpy()
        assert np.array_equal(cb, o.cb)
        c = cb & 1
        m = np.stack([c != np.roll(c, -1, axis=2), c != np.roll(c, -1, axis=1), c != np.roll(c, -1, axis=0)])
        assert np.max(np.abs(s[m] - o.s[m])) <= 1e-12
    b.close()


def _same_events(got, ref):
    """Event counters equal; the tile count depends on the tile shape."""
    return {k: v for k, v in got.items() if k != "tiles"} == {k: v for k, v in ref.items() if k != "tiles"}


def test_autotune_keeps_the_state_and_the_result():
    insts = instances(5, [24, 32, 20])
    ref = reference_states(insts, 4)
    b = make_batch(insts)
    before = [b.instance(i).get_state() for i in range(len(insts))]
    ms = b.autotune(sweeps=3)
    assert set(ms) == set(ebit.TILE_SHAPES)
    assert all(len(v) >= 1 and all(t > 0 for t in v) for v in ms.values())
    sh, dims = b.tile_shape()
    c, m = b.launch_shape()
    assert dims == ebit.TILE_SHAPES[sh] and 1 <= c <= m
    assert ms[dims][c - 1] == min(t for v in ms.values() for t in v)
    for i in range(len(insts)):
        cb, s = b.instance(i).get_state()
        assert torch.equal(cb, before[i][0]) and torch.equal(s, before[i][1])
    b.run(0, 4, graph=True)
    b.sync()
    for i, (cb_r, s_r, _, cnt_r) in enumerate(ref):
        cb, s = b.instance(i).get_state()
        assert torch.equal(cb.cpu(), cb_r) and torch.equal(s.cpu(), s_r)
        assert _same_events(b.instance(i).counters(), cnt_r)
        if sh == 0:
            assert b.instance(i).counters() == cnt_r
    b.close()


@pytest.mark.parametrize("shape", [1, 2])
def test_every_tile_shape_equals_separate_contexts(shape):
    """16x8x4 and 32x4x4 band tiles (ragged instances: 24, 20 and 40 are not
    multiples of 16 or 32) give the 8^3 result: colours, offsets, fractions
    and event counters."""
    insts = instances(4, [20, 24, 32, 40, 24])
    steps = 5
    ref = reference_states(insts, steps)
    b = make_batch(insts)
    b.set_tile_shape(shape)
    assert b.tile_shape() == (shape, ebit.TILE_SHAPES[shape])
    b.run(0, steps, graph=True)
    b.sync()
    for i, (cb_r, s_r, C_r, cnt_r) in enumerate(ref):
        g = b.instance(i)
        cb, s = g.get_state()
        assert torch.equal(cb.cpu(), cb_r), f"instance {i}: colours differ"
        assert torch.equal(s.cpu(), s_r), f"instance {i}: offsets differ"
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.front2vof(C)
        assert torch.equal(C.cpu(), C_r), f"instance {i}: volume fractions differ"
        assert _same_events(g.counters(), cnt_r), (i, g.counters(), cnt_r)
    b.close()


def test_tile_shape_changes_between_steps():
    """Re-tiling between steps (every tile marked, then the band re-formed)
    continues the same run."""
    insts = instances(12, [24, 40, 32])
    ref = reference_states(insts, 6)
    b = make_batch(insts)
    for k, shape in enumerate((0, 2, 1)):
        b.set_tile_shape(shape)
        b.run(2 * k, 2, graph=(k != 1))
    b.sync()
    for i, (cb_r, s_r, C_r, cnt_r) in enumerate(ref):
        g = b.instance(i)
        cb, s = g.get_state()
        assert torch.equal(cb.cpu(), cb_r) and torch.equal(s.cpu(), s_r)
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.front2vof(C)
        assert torch.equal(C.cpu(), C_r)
        assert _same_events(g.counters(), cnt_r)
    with pytest.raises(ebit.EbitError):
        b.set_tile_shape(len(ebit.TILE_SHAPES))
    b.close()


def test_tile_shape_that_does_not_fit_is_refused():
    """A 16-cell instance is too small for 32-cell tile edges (the staged
    region would wrap twice): refused on the host, and the autotuner skips
    that shape."""
    insts = instances(13, [16, 24])
    b = make_batch(insts)
    with pytest.raises(ebit.EbitError) as e:
        b.set_tile_shape(2)
    assert e.value.code == ebit.EBIT_EINVAL
    assert b.tile_shape()[0] == 0
    ms = b.autotune(sweeps=2)
    assert ms[(32, 4, 4)] == [] and ms[(8, 8, 8)] and ms[(16, 8, 4)]
    b.close()


def test_instance_context_refuses_its_own_sweep():
    insts = instances(6, [16])
    b = make_batch(insts)
    g = b.instance(0)
    with pytest.raises(ebit.EbitError):
        g.sweep(0, dev(insts[0][3][0]), 0.5 / 16)
    b.close()


def test_per_call_velocity_matches_stored_velocity():
    insts = instances(8, [16, 24])
    a = make_batch(insts)
    b = ebit.Batch([(n, n, n) for n, *_ in insts])
    for i, (n, phi, faces, u) in enumerate(insts):
        b.instance(i).init(dev(phi), dev(faces))
    us = [[dev(u[d]) for d in range(3)] for (_, _, _, u) in insts]
    dts = [0.5 / n for n, *_ in insts]
    for d in (0, 1, 2, 2, 1, 0):
        a.sweep(d)
        b.sweep(d, [us[i][d] for i in range(len(insts))], dts)
    a.sync()
    b.sync()
    for i in range(len(insts)):
        ca, sa = a.instance(i).get_state()
        cb_, sb = b.instance(i).get_state()
        assert torch.equal(ca, cb_) and torch.equal(sa, sb)
    a.close()
    b.close()


@pytest.mark.parametrize("graph,shape", [(True, 0), (False, 0), (True, 2)])
def test_batch_on_members_of_the_64_instance_config(graph, shape):
    """The first four instances of the batched workload itself (96^3, 128^3,
    128^3 and 64^3, their own fields and spheres, dt = 0.5 h): three steps of
    the batch against separate contexts, bit for bit, with the same counters."""
    insts = W.batched_instances(limit=4)
    assert sorted(n for n, *_ in insts) == [64, 96, 128, 128]
    steps = 3
    ref = []
    for n, phi, faces, u, dt in insts:
        g = ebit.Grid(n, n, n)
        g.init(dev(phi), dev(faces))
        ud = [dev(u[d]) for d in range(3)]
        for k in range(steps):
            g.step(k, ud, dt)
        cb, s = g.get_state()
        ref.append((cb.cpu(), s.cpu(), g.counters()))
        g.close()
    b = ebit.Batch([(n, n, n) for n, *_ in insts])
    uf = []
    for i, (n, phi, faces, u, dt) in enumerate(insts):
        b.instance(i).init(dev(phi), dev(faces))
        uf.append(tuple(dev(u[d]) for d in range(3)))
    b.set_velocity(uf, [dt for *_, dt in insts])
    b.set_tile_shape(shape)
    b.run(0, steps, graph=graph)
    b.sync()
    for i, (cb_r, s_r, cnt_r) in enumerate(ref):
        cb, s = b.instance(i).get_state()
        assert torch.equal(cb.cpu(), cb_r), f"instance {i}: colours differ"
        assert torch.equal(s.cpu(), s_r), f"instance {i}: offsets differ"
        got = b.instance(i).counters()
        assert (got == cnt_r) if shape == 0 else _same_events(got, cnt_r), (i, got, cnt_r)
        assert cnt_r["markers"] > 0
    b.close()
