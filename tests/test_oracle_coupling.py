"""Pins of the oracle's one-fluid coupling terms (oracle/coupling.py): Eq. 6 at
its end points, the well-balanced property of the face force (the force is the
backward difference of the pressure sigma kappa C when the curvature is
uniform, hence a Laplace jump of 2 sigma / R across a sphere and a zero net
force on a periodic grid), the face-curvature reading case by case, and zero
force on a plane."""
import numpy as np

import oracle
from oracle import coupling as CP
from paper_2509_26361_gb300 import workloads as W


def test_eq6_end_points_and_mixture():
    C = np.array([0.0, 1.0, 0.25, 0.5])
    rho, mu = CP.properties(C, 1000.0, 1.2, 1e-3, 1.8e-5)
    assert rho[0] == 1.2 and rho[1] == 1000.0 and mu[0] == 1.8e-5 and mu[1] == 1e-3
    assert abs(rho[2] - (250.0 + 0.9)) < 1e-12 and abs(rho[3] - 500.6) < 1e-12


def _sphere(n=24, r=0.3):
    sp = [W.Sphere((0.47, 0.52, 0.49), r)]
    n3 = (n, n, n)
    phi, faces = W.sphere_phi_nodes_faces(n3, sp)
    st = oracle.init(phi, faces, W.sphere_edge_roots(n3, sp))
    C, _ = oracle.front2vof(st)
    return C, 1.0 / n, r


def test_uniform_curvature_is_well_balanced():
    """kappa = 2/R on every interfacial cell: each face force equals the
    backward difference of p = sigma (2/R) C, so p jumps by 2 sigma / R from
    outside to inside and the forces sum to zero."""
    C, h, R = _sphere()
    sigma = 0.07
    iface = (C > 0) & (C < 1)
    kh = np.where(iface, 2.0 * h / R, 0.0)
    st = np.where(iface, 1, 0).astype(np.uint8)
    f = CP.csf_force(C, kh, st, h, sigma)
    p = sigma * (2.0 / R) * C
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        grad = (p - np.roll(p, 1, axis=ax)) / h
        assert np.abs(f[a] - grad).max() <= 1e-9 * np.abs(grad).max()
        assert abs(f[a].sum()) <= 1e-9 * np.abs(f[a]).sum()
    # the jump along the x-line through the centre, from the wall to the middle
    n = C.shape[0]
    line = f[0][n // 2, n // 2, :]
    jump = line[1:n // 2 + 1].sum() * h
    assert abs(jump - 2.0 * sigma / R) <= 1e-9 * 2.0 * sigma / R


def test_face_curvature_reading():
    h = 0.5
    st = np.array([[[1, 5, 0, 4, 2, 0]]], np.uint8)
    kh = np.array([[[0.2, 0.4, 9.0, 9.0, 0.1, 0.3]]])
    kf = CP.face_curvature(kh, st, h, 0)[0, 0]
    k = kh[0, 0] / h
    # face i lies between cells i-1 and i (periodic)
    assert kf[0] == k[0]                      # cell 5 invalid (status 0), cell 0 valid
    assert kf[1] == 0.5 * (k[0] + k[1])       # both valid (HF x and network)
    assert kf[2] == k[1]                      # cell 2 status 0
    assert kf[3] == 0.0                       # statuses 0 and 4: none valid
    assert kf[4] == k[4]                      # status 4 beside a valid cell
    assert kf[5] == k[4]                      # cell 5 status 0


def test_plane_has_no_force_and_zero_curvature_gives_zero():
    n = 16
    C = np.zeros((n, n, n))
    C[:, :, 4:10] = 1.0
    C[:, :, 10] = 0.37
    st = np.zeros(C.shape, np.uint8)
    st[:, :, 10] = 1
    f = CP.csf_force(C, np.zeros_like(C), st, 1.0 / n, 0.07)
    assert not f.any()
