"""Host-side data of the learned curvature (paper_2509_26361_gb300/curvature_data.py):
level sets, exact crossings, marker centroids and analytic labels, checked
against the closed forms and the oracle's independent routines."""
import numpy as np

import oracle
from oracle import mlp as omlp
from paper_2509_26361_gb300 import curvature_data as D
from paper_2509_26361_gb300 import workloads as W


def _ells(seed=0, n=40, count=3, amin=3.0, amax=8.0):
    return D.random_ellipsoids(np.random.default_rng(seed), count, amin, amax, n)


def test_local_level_sets_have_the_signs_of_the_global_ones():
    n = 40
    ells = _ells()
    f = D.ellipsoid_fields((n, n, n), ells)
    phi, faces = W.ellipsoid_phi_nodes_faces((n, n, n), ells)
    assert np.array_equal(f.phi >= 0, phi >= 0)
    assert np.array_equal(f.phi_faces >= 0, faces >= 0)


def test_exact_crossings_lie_on_the_surface():
    n = 40
    ells = _ells(1)
    f = D.ellipsoid_fields((n, n, n), ells)
    h = 1.0 / n
    for d in range(3):
        k, j, i = np.nonzero(np.isfinite(f.s_exact[d]))
        assert len(k) > 50
        t = f.s_exact[d][k, j, i]
        assert np.all((t >= 0) & (t <= 1))
        x = np.stack([i * h, j * h, k * h], axis=1)
        x[:, d] += t * h
        best = np.full(len(t), np.inf)
        for e in ells:
            dd = x - np.asarray(e.centre)
            dd -= np.round(dd)
            xb = dd @ np.asarray(e.rot)
            F = np.sum((xb / np.asarray(e.axes)) ** 2, axis=1) - 1.0
            best = np.minimum(best, np.abs(F))
        assert np.max(best) <= 1e-12
        # the crossing edges are exactly the sign changes of the level set
        pb = np.roll(f.phi, -1, axis=2 - d)
        assert np.array_equal((f.phi >= 0) != (pb >= 0), np.isfinite(f.s_exact[d]))


def test_nearest_point_and_curvature_agree_with_the_oracle_routines():
    rng = np.random.default_rng(3)
    axes = (0.05, 0.09, 0.13)
    p = rng.normal(scale=0.1, size=(3000, 3))
    x = D.nearest_point_on_ellipsoid(p, axes)
    assert np.max(np.abs(x - omlp.ellipsoid_closest_point(p, axes))) <= 1e-12
    k = D.ellipsoid_mean_curvature_sum(x, axes)
    assert np.max(np.abs(k - omlp.ellipsoid_mean_curvature(x, axes)) / np.abs(k)) <= 1e-12


def test_sphere_labels_are_two_over_radius_and_centroids_sit_in_their_cells():
    n = 32
    sp = W.Sphere((0.43, 0.51, 0.47), 0.2)
    e = W.Ellipsoid(sp.centre, (0.2, 0.2, 0.2), W.random_rotation(np.random.default_rng(2)))
    f = D.ellipsoid_fields((n, n, n), [e])
    st = oracle.init(D_finite(f.phi), D_finite(f.phi_faces), f.s_exact)
    C, _ = oracle.front2vof(st)
    cells = np.nonzero(((C > 0) & (C < 1)).ravel())[0]
    cent = D.interface_centroids((n, n, n), st.cb, st.s, cells)
    assert np.all(np.isfinite(cent)) and np.all((cent >= 0) & (cent <= 1))
    # centroids of markers on a sphere of radius 6.4 cells lie within a fraction of a cell of it
    i, j, k = cells % n, (cells // n) % n, cells // (n * n)
    pw = (np.stack([i, j, k], axis=1) + cent) / n - np.asarray(sp.centre)
    assert np.max(np.abs(np.linalg.norm(pw, axis=1) - 0.2) * n) <= 0.25
    lab = D.curvature_labels((n, n, n), [e], f, cent, cells)
    assert np.allclose(lab, 2.0 / (0.2 * n), rtol=1e-12, atol=0)
    lab0 = D.curvature_labels((n, n, n), [e], f, cent, cells, inside=0)
    assert np.array_equal(lab0, -lab)


def D_finite(a):
    return np.where(np.isfinite(a), a, np.sign(a))
