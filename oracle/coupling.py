"""Oracle for the one-fluid coupling terms of the EBIT interface (arxiv
2509.26361, Sec. 2.5, Eq. 6 and the surface-tension term of the momentum
equation).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. 6: the density and viscosity of the mixture are rho = H rho1 + (1 - H) rho2
and mu = H mu1 + (1 - H) mu2, with the Heaviside function H of the reference
phase approximated by the Front2VOF fraction C.

Surface tension F = sigma kappa n delta_S is discretised as a continuum surface
force on the faces of the MAC grid, from height-function curvatures, in the
well-balanced form: on the a-face between cells idx - e_a and idx,
    f_a = sigma kappa_f (C[idx] - C[idx - e_a]) / h,
the discrete gradient of C times sigma kappa_f, so that a pressure sigma kappa C
balances it exactly when kappa_f is uniform.  The paper fixes the form but not
the face curvature; the reading here: kappa = kappa_h / h of the cells whose
curvature status is valid (height functions along x, y, z or the network:
statuses 1, 2, 3, 5); on a face, the mean of its two cells' values when both
are valid, the valid one when only one is, and 0 when neither is.

Layout as in the package: arrays indexed [k, j, i] (x fastest), periodic; the
a-face of cell idx is its lower face normal to a, where u_a lives.
"""
from __future__ import annotations

import numpy as np

VALID = (1, 2, 3, 5)


def properties(C, rho1, rho2, mu1, mu2):
    """Eq. 6 with H = C, cell by cell: (rho, mu)."""
    C = np.asarray(C, np.float64)
    return C * rho1 + (1.0 - C) * rho2, C * mu1 + (1.0 - C) * mu2


def face_curvature(kh, st, h, axis):
    """kappa_f on the lower a-faces (a = axis), by the reading above."""
    ok = np.isin(np.asarray(st), VALID)
    k = np.where(ok, np.asarray(kh, np.float64) / h, 0.0)
    roll = {0: (1, 2), 1: (1, 1), 2: (1, 0)}[axis]
    kn = np.roll(k, roll[0], axis=roll[1])    # the cell idx - e_a
    okn = np.roll(ok, roll[0], axis=roll[1])
    return np.where(ok & okn, 0.5 * (k + kn), np.where(ok, k, np.where(okn, kn, 0.0)))


def csf_force(C, kh, st, h, sigma):
    """Face-centred CSF force per unit volume, shape (3, nz, ny, nx)."""
    C = np.asarray(C, np.float64)
    out = np.zeros((3,) + C.shape)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        Cn = np.roll(C, 1, axis=ax)
        kf = face_curvature(kh, st, h, a)
        out[a] = sigma * kf * (C - Cn) / h
    return out
