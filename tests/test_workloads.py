"""Seeded input generators (paper_2509_26361_gb300/workloads.py and
curvature_data.py): properties the configurations rely on, checked on the CPU."""
import numpy as np
from scipy import ndimage

from paper_2509_26361_gb300 import curvature_data as D
from paper_2509_26361_gb300 import workloads as W


def _div(u):
    """Discrete divergence of a MAC field on the unit periodic box, times h_x."""
    nz, ny, nx = u.shape[1:]
    return ((np.roll(u[0], -1, 2) - u[0]) * nx + (np.roll(u[1], -1, 1) - u[1]) * ny
            + (np.roll(u[2], -1, 0) - u[2]) * nz) / nx


def test_fourier_field_is_discretely_divergence_free_and_scaled():
    u = W.fourier_velocity((24, 20, 16), np.random.default_rng(0))
    assert np.max(np.abs(_div(u))) <= 1e-12
    assert abs(np.max(np.abs(u)) - 1.0) <= 1e-15


def test_cellular_mode_converges_on_its_centre_and_is_divergence_free():
    n = 64
    c = (0.37, 0.52)
    u = W.cellular_velocity((n, n, n), c, amp=1.0, k=2)
    assert np.max(np.abs(_div(u))) <= 1e-12
    assert np.all(u[2] == 0.0)
    # on the line y = c_y (face centres sit half a cell off the nodes), u_x points to c_x
    j = int(round(c[1] * n - 0.5))
    x = np.arange(n) / n
    near = np.abs(x - c[0]) < 0.2
    ux = u[0][0, j, :]
    assert np.all(np.sign(ux[near & (x > c[0] + 1.0 / n)]) < 0)
    assert np.all(np.sign(ux[near & (x < c[0] - 1.0 / n)]) > 0)


def test_converging_drops_start_apart_with_the_stated_gap():
    w = W.merging_drops(n=128, seed=5, amin_cells=10.0, amax_cells=20.0, gap_cells=6.0)
    lab, nc = ndimage.label(w.phi >= 0)
    assert nc == 2
    e1, e2 = w.shapes
    gap = (e2.centre[0] - W._extent(e2, 0)) - (e1.centre[0] + W._extent(e1, 0))
    assert abs(gap * 128 - 6.0) <= 1e-9
    assert np.max(np.abs(_div(w.u))) <= 1e-12
    assert np.max(np.abs(w.u)) <= 1.1 + 1e-12
    # exact crossings on exactly the sign-change edges
    for d in range(3):
        pb = np.roll(w.phi, -1, axis=2 - d)
        assert np.array_equal((w.phi >= 0) != (pb >= 0), np.isfinite(w.s_exact[d]))


def test_batched_instances_follow_the_recipe():
    insts = W.batched_instances(seed=4, count=12)
    assert len(insts) == 12
    for n, phi, faces, u, dt in insts:
        assert n in (32, 48, 64, 96, 128)
        assert phi.shape == (n, n, n) and faces.shape == (3, n, n, n) and u.shape == (3, n, n, n)
        assert dt == 0.5 / n
        lab, nc = ndimage.label(phi >= 0)
        assert 1 <= nc <= 4 + 4   # 1-4 spheres; a sphere cut by the periodic seam counts twice here
        assert np.max(np.abs(_div(u))) <= 1e-12


def test_random_ellipsoids_keep_their_gap():
    n = 96
    ells = D.random_ellipsoids(np.random.default_rng(3), 20, 3.0, 9.0, n, gap_cells=3.0)
    for i, a in enumerate(ells):
        assert all(3.0 / n - 1e-12 <= v <= 9.0 / n + 1e-12 for v in a.axes)
        assert np.allclose(np.asarray(a.rot) @ np.asarray(a.rot).T, np.eye(3), atol=1e-12)
        for b in ells[i + 1:]:
            d = np.asarray(a.centre) - np.asarray(b.centre)
            d -= np.round(d)
            assert np.linalg.norm(d) > max(a.axes) + max(b.axes) + 3.0 / n
