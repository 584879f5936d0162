"""The allocation-free sweep (ebit_advect_sweep_noalloc) against the context
sweep (ebit_advect_sweep), through the C ABI, on two calls in a row.

Callers that cannot allocate device memory -- a solver that reserves all of its
device memory at start-up, a real-time loop where cudaMalloc may not run -- use
the allocation-free entry point; it must give the same state as the regular
one.  This file is collected last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _present(cb):
    c = cb & 1
    return np.stack([c != np.roll(c, -1, 2), c != np.roll(c, -1, 1), c != np.roll(c, -1, 0)])


@pytest.mark.parametrize("n", [32, 40])
def test_noalloc_sweep_matches_context_sweep_twice(n):
    w = W.fourier_spheres(n=n, seed=3, count=4, rmin=0.08, rmax=0.16, steps=2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = ebit.Grid(n, n, n)
    g.init(dev(w.phi), dev(w.phi_faces))
    cb, s = g.get_state()
    ud = [dev(w.u[d]) for d in range(3)]
    cb_a, s_a = cb.clone(), s.clone()
    cb_b, s_b = torch.empty_like(cb), torch.empty_like(s)
    for k, d in enumerate((0, 1)):  # two calls in a row, each fed the previous output
        dt = (0.8 if k == 0 else -0.6) * g.h
        g.sweep(d, ud[d], dt)
        code = ebit.ebit_advect_sweep_noalloc(w.n3, g.h, d, cb_a, s_a, ud[d], dt, cb_b, s_b)
        assert code == ebit.EBIT_OK
        torch.cuda.synchronize()
        ref_cb, ref_s = g.get_state()
        got_cb, got_s = cb_b.cpu().numpy(), s_b.cpu().numpy()
        ref_cb, ref_s = ref_cb.cpu().numpy(), ref_s.cpu().numpy()
        assert np.array_equal(got_cb, ref_cb)
        m = _present(ref_cb)
        assert np.abs(got_s[m] - ref_s[m]).max() <= TOL
        assert np.all(got_s[~m] == 0.0)
        cb_a, s_a, cb_b, s_b = cb_b, s_b, cb_a, s_a
    g.close()


def _cell_spheres(n3, rng, count):
    """Level set of a few spheres measured in cells (radii 2.5-4 cells, periodic),
    at the nodes and at the three families of face centres."""
    nx, ny, nz = n3
    cs = [rng.uniform(0, n3) for _ in range(count)]
    rs = rng.uniform(2.5, 4.0, count)

    def phi_at(sh):
        x = np.arange(nx) + sh[0]
        y = np.arange(ny) + sh[1]
        z = np.arange(nz) + sh[2]
        out = np.full((nz, ny, nx), -np.inf)
        for c, r in zip(cs, rs):
            d = [v - cc for v, cc in zip((x, y, z), c)]
            d = [dd - n * np.round(dd / n) for dd, n in zip(d, n3)]
            q = d[0][None, None, :] ** 2 + d[1][None, :, None] ** 2 + d[2][:, None, None] ** 2
            out = np.maximum(out, r * r - q)
        return out

    faces = np.stack([phi_at((0, 0.5, 0.5)), phi_at((0.5, 0, 0.5)), phi_at((0.5, 0.5, 0))])
    return phi_at((0, 0, 0)), faces


@pytest.mark.parametrize("n3", [(20, 24, 36), (60, 60, 72), (9, 9, 3236)])
def test_noalloc_ragged_grids_with_many_tiles(n3):
    """Axes that are not multiples of the 8-cell tile: 60 x 60 x 72 has 576
    tiles and 9 x 9 x 3236 has 1620, the most any grid of at most 64^3 cells
    can have.  Two calls in a row against the context sweep."""
    rng = np.random.default_rng(sum(n3))
    nx, ny, nz = n3
    phi, faces = _cell_spheres(n3, rng, 6 if nz < 1000 else 40)
    u = W.fourier_velocity(n3, rng)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = ebit.Grid(nx, ny, nz, h=1.0 / nx)
    g.init(dev(phi), dev(faces))
    cb, s = g.get_state()
    ud = [dev(u[d]) for d in range(3)]
    cb_a, s_a = cb.clone(), s.clone()
    cb_b, s_b = torch.empty_like(cb), torch.empty_like(s)
    for k, d in enumerate((2, 0)):
        dt = (0.7 if k == 0 else -0.5) * g.h
        g.sweep(d, ud[d], dt)
        assert ebit.ebit_advect_sweep_noalloc(n3, g.h, d, cb_a, s_a, ud[d], dt, cb_b, s_b) == ebit.EBIT_OK
        torch.cuda.synchronize()
        ref_cb, ref_s = (t.cpu().numpy() for t in g.get_state())
        got_cb, got_s = cb_b.cpu().numpy(), s_b.cpu().numpy()
        assert np.array_equal(got_cb, ref_cb)
        m = _present(ref_cb)
        assert m.any()
        assert np.abs(got_s[m] - ref_s[m]).max() <= TOL
        assert np.all(got_s[~m] == 0.0)
        cb_a, s_a, cb_b, s_b = cb_b, s_b, cb_a, s_a
    g.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    n3 = (80, 64, 64)
    N = 80 * 64 * 64
    cb = torch.zeros(N, dtype=torch.uint8, device="cuda")
    s = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(ebit.EbitError) as e:
        ebit.ebit_advect_sweep_noalloc(n3, 1.0 / 80, 0, cb, s, u, 0.001, cb.clone(), s.clone())
    assert e.value.code == ebit.EBIT_EINVAL
