"""AMR refinement rule and narrow-band brick store (Sec. 2.5) on the CUDA path,
through the C ABI: the refinement mask equals the oracle's on evolved states
(ragged grids included), the bricks are the oracle's tiles, and a state packed
into the store and unpacked into a fresh context is the same state bit for
bit and steps on identically."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import amr
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _evolved(n3, seed, steps):
    rng = np.random.default_rng(seed)
    rmin = 2.5 / min(n3)
    sp = W.random_spheres(rng, 1 if min(n3) < 16 else 3, rmin, max(0.2, rmin + 0.05), min(n3))
    phi, faces = W.sphere_phi_nodes_faces(n3, sp)
    u = [dev(v) for v in W.fourier_velocity(n3, rng)]
    g = ebit.Grid(*n3)
    g.init(dev(phi), dev(faces))
    for k in range(steps):
        g.step(k, u, 0.6 * g.h)
    return g, u


@pytest.mark.parametrize("n3,seed,steps", [((32, 32, 32), 1, 3), ((20, 24, 28), 2, 4), ((9, 17, 8), 3, 2)])
def test_refine_mask_matches_the_oracle(n3, seed, steps):
    g, _ = _evolved(n3, seed, steps)
    cb, _ = g.get_state()
    mask, count = g.refine_mask()
    ref = amr.refine_mask(cb.cpu().numpy())
    assert np.array_equal(mask.cpu().numpy().astype(bool), ref)
    assert count == int(ref.sum()) and 0 < count <= np.prod(n3)
    g.close()


@pytest.mark.parametrize("n3,seed", [((32, 32, 32), 4), ((20, 24, 28), 5)])
def test_brick_store_round_trip(n3, seed):
    g, u = _evolved(n3, seed, 3)
    cb, s = g.get_state()
    st = g.pack_bricks()
    assert np.array_equal(st["tiles"].cpu().numpy(), amr.brick_tiles(cb.cpu().numpy()))
    assert 0 < st["tiles"].numel() <= g.tiles
    h = ebit.Grid(*n3)
    h.unpack_bricks(st)
    cb2, s2 = h.get_state()
    assert torch.equal(cb2, cb) and torch.equal(s2, s)
    # both continue identically, Front2VOF included
    for k in range(3, 5):
        g.step(k, u, 0.6 * g.h)
        h.step(k, u, 0.6 * h.h)
    a, b = g.get_state(), h.get_state()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    Ca = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    Cb = torch.zeros_like(Ca)
    g.front2vof(Ca, ebit.EBIT_FULL)
    h.front2vof(Cb, ebit.EBIT_FULL)
    assert torch.equal(Ca, Cb)
    g.close()
    h.close()


def test_uniform_domain_has_no_bricks():
    n3 = (16, 16, 16)
    g = ebit.Grid(*n3)
    phi = np.full((n3[2], n3[1], n3[0]), -1.0)
    faces = np.full((3,) + phi.shape, -1.0)
    g.init(dev(phi), dev(faces))
    st = g.pack_bricks()
    assert st["tiles"].numel() == 0 and int(st["bg"].sum()) == 0
    mask, count = g.refine_mask()
    assert count == 0 and int(mask.sum()) == 0
    h = ebit.Grid(*n3)
    h.unpack_bricks({"tiles": st["tiles"], "cb": st["cb"], "s": st["s"], "bg": st["bg"] | 1})
    cb, s = h.get_state()
    assert bool((cb == 0x0F).all()) and float(s.abs().max()) == 0.0
    g.close()
    h.close()


def test_refusals():
    n3 = (24, 16, 16)
    g, _ = _evolved(n3, 6, 1)
    lib = ebit.load()
    n = ctypes.c_int()
    assert lib.ebit_pack_bricks(g.ctx, 0, None, None, None, None, ctypes.byref(n)) == ebit.EBIT_OK and n.value > 1
    cap = n.value - 1
    t = torch.empty(cap, dtype=torch.int32, device="cuda")
    cb = torch.empty((cap, 512), dtype=torch.uint8, device="cuda")
    s = torch.empty((cap, 3, 512), dtype=torch.float64, device="cuda")
    bg = torch.empty(g.tiles, dtype=torch.uint8, device="cuda")
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    assert lib.ebit_pack_bricks(g.ctx, cap, P(t), P(cb), P(s), P(bg), ctypes.byref(n)) == ebit.EBIT_EINVAL
    st = g.pack_bricks()
    bad = dict(st)
    bad["tiles"] = st["tiles"].clone()
    bad["tiles"][0] = g.tiles  # one past the last tile
    with pytest.raises(ebit.EbitError) as e:
        g.unpack_bricks(bad)
    assert e.value.code == ebit.EBIT_EINVAL
    g.close()
