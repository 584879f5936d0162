"""Training and evaluation data of the learned curvature (host side).

The learned curvature maps the 3x3x3 volume-fraction stencil of an interface
cell to kappa*h.  Its data are made the way the method makes fractions: seeded
ellipsoids (spheres included) are sampled as level sets, markers are placed on
the edges at the exact surface crossings, Front2VOF (Sec. 2.5, Eq. 7) turns them
into fractions on the GPU, and the encoded canonical stencils are gathered on
the GPU.  The label of a cell is the analytic mean-curvature sum of its
ellipsoid at the surface point nearest the cell's interface centroid (the mean
of the markers on the cell's edges), times h.  Everything here is analytic
geometry on the host; the fractions and stencils come from the CUDA library.

Units: domain [0, 1)^3, n cells per axis, h = 1/n.  Arrays are indexed [k, j, i].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .workloads import Ellipsoid, random_rotation


# ------------------------------------------------------------------ shapes
def random_ellipsoids(rng, count, amin_cells, amax_cells, n, gap_cells=3.0, log_uniform=False,
                      sphere_fraction=0.0, tries=200000):
    """``count`` non-overlapping ellipsoids with semi-axes in [amin, amax] cells
    (uniform, or log-uniform), uniform random rotations, a ``sphere_fraction``
    of them spheres.  Bounding spheres keep ``gap_cells`` apart (periodic), and
    the larger shapes are placed first."""
    h = 1.0 / n

    def draw(size):
        if log_uniform:
            return np.exp(rng.uniform(np.log(amin_cells), np.log(amax_cells), size=size))
        return rng.uniform(amin_cells, amax_cells, size=size)

    axes = []
    for _ in range(count):
        if rng.uniform() < sphere_fraction:
            axes.append(np.full(3, draw(1)[0]))
        else:
            axes.append(draw(3))
    order = np.argsort([-a.max() for a in axes])
    placed = []
    cen = np.zeros((count, 3))
    rad = np.zeros(count)
    for idx in order:
        a = axes[idx] * h
        rb = a.max()
        np_ = len(placed)
        for _ in range(tries):
            c = rng.uniform(0.0, 1.0, size=3)
            d = cen[:np_] - c
            d -= np.round(d)
            if np_ == 0 or np.all(np.sqrt(np.sum(d * d, axis=1)) > rb + rad[:np_] + gap_cells * h):
                placed.append(Ellipsoid(tuple(float(v) for v in c), tuple(float(v) for v in a),
                                        random_rotation(rng)))
                cen[np_] = c
                rad[np_] = rb
                break
        else:
            raise RuntimeError("could not place the requested ellipsoids")
    return placed


@dataclass
class Fields:
    phi: np.ndarray        # (nz, ny, nx) level set at the nodes, > 0 inside
    phi_faces: np.ndarray  # (3, nz, ny, nx) at the face centres
    s_exact: np.ndarray    # (3, nz, ny, nx) exact crossing offsets, NaN elsewhere
    owner: np.ndarray      # (nz, ny, nx) int32: ellipsoid of largest phi near the node, -1 far away


def _box(c, r, n):
    """Unwrapped node indices covering [c - r, c + r] (domain units) on one axis."""
    lo = int(np.floor((c - r) * n)) - 1
    hi = int(np.ceil((c + r) * n)) + 2
    return np.arange(lo, hi)


def ellipsoid_fields(n3, ells, inside=1):
    """Level set 1 - |A^-1 R^T (x - c)|^2 of every ellipsoid, evaluated in a
    local box around it (periodic) and combined by max; exact edge crossings of
    the quadratic along each edge; the owning ellipsoid per node.  With
    ``inside=0`` the phases swap (phi -> -phi: phase 1 outside, bubbles)."""
    nx, ny, nz = n3
    if not (nx == ny == nz):
        raise ValueError("cubic grids only")
    n = nx
    h = 1.0 / n
    phi = np.full((nz, ny, nx), -np.inf)
    phif = np.full((3, nz, ny, nx), -np.inf)
    s_ex = np.full((3, nz, ny, nx), np.nan)
    owner = np.full((nz, ny, nx), -1, dtype=np.int32)
    shifts = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))
    for k, e in enumerate(ells):
        c = np.asarray(e.centre)
        a = np.asarray(e.axes)
        R = np.asarray(e.rot)
        rb = a.max() + 2.0 * h
        bi = [_box(c[d], rb, n) for d in range(3)]  # x, y, z unwrapped indices

        def level(sh):
            dx = (bi[0] + sh[0]) * h - c[0]
            dy = (bi[1] + sh[1]) * h - c[1]
            dz = (bi[2] + sh[2]) * h - c[2]
            v = np.ones((len(bi[2]), len(bi[1]), len(bi[0])))
            for b in range(3):
                xb = R[0, b] * dx[None, None, :] + R[1, b] * dy[None, :, None] + R[2, b] * dz[:, None, None]
                v -= (xb / a[b]) ** 2
            return v

        ix = np.ix_(bi[2] % nz, bi[1] % ny, bi[0] % nx)
        v = level((0.0, 0.0, 0.0))
        cur = phi[ix]
        own = owner[ix]
        own[v > cur] = k
        owner[ix] = own
        phi[ix] = np.maximum(cur, v)
        for f in range(3):
            vf = level(shifts[f])
            phif[f][ix] = np.maximum(phif[f][ix], vf)
        # exact crossings: F(t) = 1 - sum_b (q_b + t h R[d, b])^2 / a_b^2, t in [0, 1]
        for d in range(3):
            sl0 = [slice(None)] * 3
            sl1 = [slice(None)] * 3
            ax = 2 - d
            sl0[ax] = slice(0, -1)
            sl1[ax] = slice(1, None)
            v0 = v[tuple(sl0)]
            v1 = v[tuple(sl1)]
            cross = (v0 >= 0) != (v1 >= 0)
            if not np.any(cross):
                continue
            kk, jj, ii = np.nonzero(cross)
            px = bi[0][ii] * h - c[0]
            py = bi[1][jj] * h - c[1]
            pz = bi[2][kk] * h - c[2]
            q = [R[0, b] * px + R[1, b] * py + R[2, b] * pz for b in range(3)]
            A = -sum((h * R[d, b] / a[b]) ** 2 for b in range(3))
            B = -2.0 * sum(q[b] * h * R[d, b] / a[b] ** 2 for b in range(3))
            C0 = 1.0 - sum((q[b] / a[b]) ** 2 for b in range(3))
            disc = np.maximum(B * B - 4.0 * A * C0, 0.0)
            sq = np.sqrt(disc)
            # A < 0: the quadratic is concave; exactly one root in [0, 1] on a sign change
            r1 = (-B + sq) / (2.0 * A)
            r2 = (-B - sq) / (2.0 * A)
            t = np.where((r1 >= 0.0) & (r1 <= 1.0), r1, r2)
            t = np.clip(t, 0.0, 1.0)
            gi = (bi[2][kk] % nz, bi[1][jj] % ny, bi[0][ii] % nx)
            s_ex[d][gi] = t
    if inside == 0:
        phi = -phi
        phif = -phif
    return Fields(phi, phif, s_ex, owner)


# ------------------------------------------------------------------ labels
def interface_centroids(n3, cb, s, cells):
    """Mean of the markers on the 12 edges of each cell (cell units, unwrapped
    around the cell's lowest node).  cb: node colour bytes (bit 0 the node
    colour), s: (3, N) offsets, cells: linear cell ids.  Cells without markers
    get NaN."""
    nx, ny, nz = n3
    cells = np.asarray(cells, dtype=np.int64)
    i = cells % nx
    j = (cells // nx) % ny
    k = cells // (nx * ny)
    col = (np.asarray(cb).reshape(-1) & 1).astype(np.int8)
    s = np.asarray(s).reshape(3, -1)

    def lid(a, b, c):
        return ((c % nz) * ny + (b % ny)) * nx + (a % nx)

    acc = np.zeros((len(cells), 3))
    cnt = np.zeros(len(cells))
    for d in range(3):
        t1, t2 = [(1, 2), (0, 2), (0, 1)][d]
        for o1 in (0, 1):
            for o2 in (0, 1):
                off = [0, 0, 0]
                off[t1] = o1
                off[t2] = o2
                n0 = lid(i + off[0], j + off[1], k + off[2])
                e = [0, 0, 0]
                e[d] = 1
                n1 = lid(i + off[0] + e[0], j + off[1] + e[1], k + off[2] + e[2])
                has = col[n0] != col[n1]
                p = np.stack([np.full(len(cells), float(off[0])), np.full(len(cells), float(off[1])),
                              np.full(len(cells), float(off[2]))], axis=1)
                p[:, d] += s[d][n0]
                acc += np.where(has[:, None], p, 0.0)
                cnt += has
    with np.errstate(invalid="ignore", divide="ignore"):
        return acc / cnt[:, None]


def nearest_point_on_ellipsoid(p, axes, iters=80):
    """Nearest point of the ellipsoid sum (x_i / a_i)^2 = 1 to each body-frame
    point p.  The nearest point is x_i = a_i^2 p_i / (a_i^2 + t) with t the root
    of g(t) = sum (a_i p_i / (a_i^2 + t))^2 - 1 on t > -min a_i^2, where g falls
    monotonically.  Newton's method from the right of the root (g convex there)
    converges from above; a bracket guards the degenerate cases."""
    a2 = np.asarray(axes, dtype=np.float64) ** 2
    p = np.asarray(p, dtype=np.float64)
    ap = np.sqrt(a2) * p
    lo = np.full(p.shape[0], -a2.min())
    # upper start: |p| * max a bounds sqrt(sum (a_i p_i)^2) >= a_i^2 + t at the root
    t = np.sqrt(np.sum(ap * ap, axis=1)) - a2.min() + 1e-300
    t = np.maximum(t, lo + 1e-12 * a2.max())
    for _ in range(iters):
        den = a2 + t[:, None]
        r = ap / den
        g = np.sum(r * r, axis=1) - 1.0
        dg = -2.0 * np.sum(r * r / den, axis=1)
        step = g / dg
        tn = t - step
        # keep inside the domain of g: halve toward the lower bound if overshooting
        tn = np.where(tn <= lo, 0.5 * (t + lo), tn)
        t = tn
    return a2 * p / (a2 + t[:, None])


def ellipsoid_mean_curvature_sum(x, axes):
    """kappa_1 + kappa_2 of the ellipsoid at body-frame surface points x, from
    the implicit form F = sum (x_i / a_i)^2 - 1: (|grad F|^2 tr H - grad F^T H
    grad F) / |grad F|^3 with H = diag(2 / a_i^2); positive on the convex side."""
    a2 = np.asarray(axes, dtype=np.float64) ** 2
    g = 2.0 * np.asarray(x) / a2
    hd = 2.0 / a2
    gg = np.sum(g * g, axis=1)
    return (gg * hd.sum() - np.sum(g * g * hd, axis=1)) / gg ** 1.5


def curvature_labels(n3, ells, fields, centroids, cells, inside=1):
    """kappa*h at the nearest surface point of each cell's owning ellipsoid
    (sign: positive when phase 1 is the convex side)."""
    nx, ny, nz = n3
    h = 1.0 / nx
    cells = np.asarray(cells, dtype=np.int64)
    i = cells % nx
    j = (cells // nx) % ny
    k = cells // (nx * ny)
    own = fields.owner.reshape(-1)[cells]
    out = np.full(len(cells), np.nan)
    pw = np.stack([(i + centroids[:, 0]) * h, (j + centroids[:, 1]) * h, (k + centroids[:, 2]) * h], axis=1)
    for e_id in np.unique(own):
        if e_id < 0:
            continue
        sel = own == e_id
        e = ells[e_id]
        d = pw[sel] - np.asarray(e.centre)
        d -= np.round(d)
        pb = d @ np.asarray(e.rot)  # body frame: R^T d, rows
        x = nearest_point_on_ellipsoid(pb, e.axes)
        out[sel] = ellipsoid_mean_curvature_sum(x, e.axes) * h
    return out if inside else -out
