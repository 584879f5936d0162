"""Seeded synthetic inputs for the EBIT kinematics path (no method arithmetic here).

This module produces analytic shapes and velocity fields only: level sets of
spheres and ellipsoids sampled at grid nodes and face centres, exact edge/sphere
intersection offsets, and discretely divergence-free MAC velocity fields.  Both
the CUDA path and the CPU oracle consume these arrays; neither one's arithmetic
lives here.

Coordinates: unit-cube domain ``[0,1)^3`` with ``n`` cells per axis (``h = 1/n``),
node ``(i,j,k)`` at ``(i h, j h, k h)``.  Arrays are indexed ``[k, j, i]``.  Face
arrays ``(3, nz, ny, nx)``: entry ``[a, k, j, i]`` belongs to the face normal to
axis ``a`` whose lowest corner is node ``(i,j,k)``; its centre is the node shifted
by ``h/2`` along the two other axes.  A velocity component ``u_a`` lives on the
a-normal faces.

The workloads mirror the paper's kinematic tests (translation of a sphere,
Sec. 3.1; deformation-type divergence-free flow, Sec. 3.2) at the sizes of the
benchmark configurations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _grid(n3):
    nx, ny, nz = n3
    x = np.arange(nx, dtype=np.float64) / nx
    y = np.arange(ny, dtype=np.float64) / ny
    z = np.arange(nz, dtype=np.float64) / nz
    return x, y, z


def _periodic_delta(a: np.ndarray, c: float) -> np.ndarray:
    """Minimum-image difference a - c on the unit period."""
    d = a - c
    return d - np.round(d)


@dataclass
class Sphere:
    centre: tuple
    radius: float
    inside: int = 1  # 1: phase 1 inside (a drop), 0: phase 1 outside


def sphere_phi(n3, spheres, shift=(0.0, 0.0, 0.0)):
    """phi = max_k (R_k^2 - |x - c_k|^2) on the lattice shifted by ``shift`` (in cells).
    Periodic minimum image.  Positive inside any sphere."""
    nx, ny, nz = n3
    x, y, z = _grid(n3)
    x = x + shift[0] / nx
    y = y + shift[1] / ny
    z = z + shift[2] / nz
    phi = np.full((nz, ny, nx), -np.inf)
    for sp in spheres:
        dx = _periodic_delta(x, sp.centre[0])[None, None, :]
        dy = _periodic_delta(y, sp.centre[1])[None, :, None]
        dz = _periodic_delta(z, sp.centre[2])[:, None, None]
        v = sp.radius * sp.radius - (dx * dx + dy * dy + dz * dz)
        phi = np.maximum(phi, v)
    return phi


def sphere_phi_nodes_faces(n3, spheres):
    """Level set at the nodes and at the three families of face centres."""
    phi = sphere_phi(n3, spheres)
    faces = np.stack([
        sphere_phi(n3, spheres, (0.0, 0.5, 0.5)),
        sphere_phi(n3, spheres, (0.5, 0.0, 0.5)),
        sphere_phi(n3, spheres, (0.5, 0.5, 0.0)),
    ])
    return phi, faces


def sphere_edge_roots(n3, spheres):
    """Exact offset (fraction of h from the lower node) of the sphere surface on
    every edge whose end signs differ; NaN elsewhere.  Shape (3, nz, ny, nx)."""
    nx, ny, nz = n3
    ns = (nx, ny, nz)
    phi = sphere_phi(n3, spheres)
    out = np.full((3,) + phi.shape, np.nan)
    x, y, z = _grid(n3)
    coords = (x[None, None, :] + 0 * phi, y[None, :, None] + 0 * phi, z[:, None, None] + 0 * phi)
    for a in range(3):
        phi_b = np.roll(phi, -1, axis=2 - a)
        cross = (phi >= 0) != (phi_b >= 0)
        idx = np.nonzero(cross)
        vals = np.full(len(idx[0]), np.nan)
        for sp in spheres:
            # offsets of the node from the centre along the three axes (min image)
            d = [_periodic_delta(coords[b][idx], sp.centre[b]) for b in range(3)]
            rest = sum(d[b] * d[b] for b in range(3) if b != a)
            disc = sp.radius * sp.radius - rest
            ok = disc >= 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            h = 1.0 / ns[a]
            for sign in (-1.0, 1.0):
                t = (sign * sq - d[a]) / h  # root position in cells from the node
                good = ok & (t >= 0.0) & (t <= 1.0) & np.isnan(vals)
                vals = np.where(good, t, vals)
        out[a][idx] = vals
    return out


def random_spheres(rng, count, rmin, rmax, n, min_gap_cells=2.0, box=(0.0, 1.0), tries=100000):
    """Non-overlapping spheres (periodic): centre gap > R1 + R2 + min_gap_cells*h."""
    h = 1.0 / n
    out = []
    for _ in range(tries):
        if len(out) == count:
            break
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(box[0], box[1], size=3)
        ok = True
        for sp in out:
            d = _periodic_delta(c, np.array(sp.centre))
            if np.sqrt(np.sum(d * d)) <= r + sp.radius + min_gap_cells * h:
                ok = False
                break
        if ok:
            out.append(Sphere(tuple(float(v) for v in c), float(r)))
    if len(out) != count:
        raise RuntimeError("could not place the requested spheres")
    return out


# --------------------------------------------------------------- ellipsoids
@dataclass
class Ellipsoid:
    centre: tuple
    axes: tuple   # semi-axes (domain units)
    rot: np.ndarray = field(default_factory=lambda: np.eye(3))  # body -> world


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid_phi(n3, ells, shift=(0.0, 0.0, 0.0)):
    """phi = max_k (1 - sum_i (x'_i / a_i)^2) (body coordinates x' = R^T (x - c))."""
    nx, ny, nz = n3
    x, y, z = _grid(n3)
    x = x + shift[0] / nx
    y = y + shift[1] / ny
    z = z + shift[2] / nz
    phi = np.full((nz, ny, nx), -np.inf)
    for e in ells:
        dx = _periodic_delta(x, e.centre[0])[None, None, :]
        dy = _periodic_delta(y, e.centre[1])[None, :, None]
        dz = _periodic_delta(z, e.centre[2])[:, None, None]
        v = np.ones((nz, ny, nx))
        for b in range(3):
            xb = e.rot[0, b] * dx + e.rot[1, b] * dy + e.rot[2, b] * dz
            v = v - (xb / e.axes[b]) ** 2
        phi = np.maximum(phi, v)
    return phi


def ellipsoid_phi_nodes_faces(n3, ells):
    phi = ellipsoid_phi(n3, ells)
    faces = np.stack([
        ellipsoid_phi(n3, ells, (0.0, 0.5, 0.5)),
        ellipsoid_phi(n3, ells, (0.5, 0.0, 0.5)),
        ellipsoid_phi(n3, ells, (0.5, 0.5, 0.0)),
    ])
    return phi, faces


# --------------------------------------------------------- velocity fields
def gyroid_surface(n, waves, phases, c0, shift=0.0, axis=0):
    """A gyroid-type triply periodic surface on an n^3 grid (cell units):
    phi = sin X cos Y + sin Y cos Z + sin Z cos X + c0 with X = 2 pi waves[0] x / n
    + phases[0] (and likewise Y, Z), moved by `shift` cells along `axis`.  Its
    product terms give faces whose diagonal corners lie on the same side (saddle
    faces), which a sum of one-axis terms never does.  Returns phi at the nodes,
    phi at the three families of face centres, and the exact offsets of the
    surface on the sign-change edges (bisection to 2^-60; NaN elsewhere)."""
    k = [2.0 * np.pi * w / n for w in waves]
    off = [0.0, 0.0, 0.0]
    off[axis] = shift

    def surf(x, y, z):
        X = k[0] * (x - off[0]) + phases[0]
        Y = k[1] * (y - off[1]) + phases[1]
        Z = k[2] * (z - off[2]) + phases[2]
        return np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X) + c0

    g = np.arange(n, dtype=np.float64)

    def at(ox, oy, oz):
        return surf(g[None, None, :] + ox, g[None, :, None] + oy, g[:, None, None] + oz)

    phi = at(0.0, 0.0, 0.0)
    faces = np.stack([at(0.0, 0.5, 0.5), at(0.5, 0.0, 0.5), at(0.5, 0.5, 0.0)])
    roots = np.full((3,) + phi.shape, np.nan)
    for a in range(3):
        cross = (phi >= 0) != (np.roll(phi, -1, axis=2 - a) >= 0)
        kk, jj, ii = np.nonzero(cross)
        base = [ii.astype(np.float64), jj.astype(np.float64), kk.astype(np.float64)]
        lo, hi = np.zeros(len(ii)), np.ones(len(ii))

        def along(t):
            p = [b.copy() for b in base]
            p[a] = p[a] + t
            return surf(p[0], p[1], p[2])

        f0 = along(lo) >= 0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            same = (along(mid) >= 0) == f0
            lo = np.where(same, mid, lo)
            hi = np.where(same, hi, mid)
        roots[a][kk, jj, ii] = 0.5 * (lo + hi)
    return phi, faces, roots


def uniform_velocity(n3, u=(1.0, 1.0, 1.0)):
    nx, ny, nz = n3
    return np.stack([np.full((nz, ny, nx), float(u[a])) for a in range(3)])


def fourier_velocity(n3, rng, modes=12, kmax=3):
    """Divergence-free MAC field from a random vector potential.

    A = sum_m amp_m sin(2 pi k_m . x + phase_m) with integer wavevectors
    1 <= |k|_inf and |k| <= kmax, sampled at edge midpoints; u = discrete curl of
    A on the faces (so the discrete divergence vanishes up to rounding), scaled so
    that max |u| = 1.  Returns shape (3, nz, ny, nx).
    """
    nx, ny, nz = n3
    cand = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(-kmax, kmax + 1):
                k = np.array([kx, ky, kz])
                if np.max(np.abs(k)) >= 1 and np.sqrt(np.sum(k * k)) <= kmax:
                    cand.append(k)
    cand = np.array(cand)
    sel = cand[rng.choice(len(cand), size=modes, replace=False)]
    amps = rng.normal(size=(modes, 3))
    phases = rng.uniform(0, 2 * np.pi, size=modes)
    x, y, z = _grid(n3)
    hs = (1.0 / nx, 1.0 / ny, 1.0 / nz)

    def potential(comp, off):
        # A_comp sampled at node + off (in cells): each mode's sine is the
        # imaginary part of a product of three 1-D complex exponentials
        v = np.zeros((nz, ny, nx), dtype=np.complex128)
        for m in range(modes):
            ex = np.exp(2j * np.pi * sel[m, 0] * (x + off[0] * hs[0]))
            ey = np.exp(2j * np.pi * sel[m, 1] * (y + off[1] * hs[1]))
            ez = np.exp(2j * np.pi * sel[m, 2] * (z + off[2] * hs[2])) * (amps[m, comp] * np.exp(1j * phases[m]))
            v += (ez[:, None, None] * ey[None, :, None]) * ex[None, None, :]
        return v.imag

    Ax = potential(0, (0.5, 0.0, 0.0))  # x-edge midpoints
    Ay = potential(1, (0.0, 0.5, 0.0))
    Az = potential(2, (0.0, 0.0, 0.5))

    def fwd(a, axis):  # a(node + e_axis) - a(node), periodic; axis in array order
        return np.roll(a, -1, axis=axis) - a

    # array axes: 0 = z, 1 = y, 2 = x
    ux = fwd(Az, 1) / hs[1] - fwd(Ay, 0) / hs[2]
    uy = fwd(Ax, 0) / hs[2] - fwd(Az, 2) / hs[0]
    uz = fwd(Ay, 2) / hs[0] - fwd(Ax, 1) / hs[1]
    u = np.stack([ux, uy, uz])
    return u / np.max(np.abs(u))


def deformation_velocity(n3):
    """LeVeque/Enright 3D deformation field (Sec. 3.2) on the MAC faces, without the
    time factor."""
    nx, ny, nz = n3
    x, y, z = _grid(n3)
    hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    X = x[None, None, :]
    Y = y[None, :, None]
    Z = z[:, None, None]
    s = np.sin
    pi = np.pi
    ux = 2 * s(pi * X) ** 2 * s(2 * pi * (Y + hy / 2)) * s(2 * pi * (Z + hz / 2))
    uy = -s(2 * pi * (X + hx / 2)) * s(pi * Y) ** 2 * s(2 * pi * (Z + hz / 2))
    uz = -s(2 * pi * (X + hx / 2)) * s(2 * pi * (Y + hy / 2)) * s(pi * Z) ** 2
    shp = (nz, ny, nx)
    return np.stack([np.broadcast_to(ux, shp), np.broadcast_to(uy, shp), np.broadcast_to(uz, shp)]).copy()


# -------------------------------------------------------------- workloads
@dataclass
class Workload:
    name: str
    n3: tuple
    phi: np.ndarray
    phi_faces: np.ndarray
    u: np.ndarray                 # (3, nz, ny, nx), max|u| = 1 unless stated
    cfl: float                    # dt = cfl * h / max|u|
    steps: int
    period: float | None = None   # cos(pi t / T) factor when set
    s_exact: np.ndarray | None = None
    shapes: list = field(default_factory=list)

    @property
    def h(self):
        return 1.0 / self.n3[0]

    def lam(self, step: int) -> float:
        """dt/h for step ``step`` with the time factor at mid-step folded in."""
        base = self.cfl
        if self.period is None:
            return base
        dt = self.cfl * self.h
        t_mid = (step + 0.5) * dt
        return base * float(np.cos(np.pi * t_mid / self.period))


def grazing_free(centre_cells, radius_cells, n, cfl, margin=1e-6):
    """True if, at every sub-step position of a uniform (1,1,1) translation with the
    given CFL (x-y-z sweeps, then z-y-x), no grid line along any axis meets the
    sphere in a chord whose two ends lie on the same edge, and no chord end lies
    within ``margin`` cells of a node."""
    sub = int(round(1.0 / cfl))
    shifts = []
    sft = np.zeros(3)
    for step in range(2 * sub):
        order = (0, 1, 2) if step % 2 == 0 else (2, 1, 0)
        for d in order:
            sft = sft.copy()
            sft[d] += cfl
            shifts.append(sft)
    lines = np.arange(n, dtype=np.float64)
    r2 = radius_cells * radius_cells
    for sft in shifts:
        c = np.asarray(centre_cells) + sft
        for a in range(3):
            b, e = [x for x in range(3) if x != a]
            db = lines[:, None] - c[b]
            de = lines[None, :] - c[e]
            db -= np.round(db / n) * n
            de -= np.round(de / n) * n
            rho2 = db * db + de * de
            hit = rho2 < r2
            half = np.sqrt(np.where(hit, r2 - rho2, 0.0))
            lo = c[a] - half
            hi = c[a] + half
            same = hit & (np.floor(lo) == np.floor(hi))
            near = hit & ((np.abs(lo - np.round(lo)) < margin) | (np.abs(hi - np.round(hi)) < margin))
            if np.any(same) or np.any(near):
                return False
    return True


def translation_sphere(n=32, seed=1, cfl=0.25, steps=128, exact=True, radius=0.15):
    """One sphere R = 0.15 at a seeded centre in [0.3, 0.7]^3, uniform u = (1,1,1)
    on a periodic n^3 grid (the paper's translation test, Sec. 3.1, periodic).

    Centres are drawn from the seeded generator until one leaves every grid line
    either well inside or well outside the sphere at all sub-step positions: a
    line that grazes the sphere has a chord shorter than a cell, whose two
    markers the one-marker-per-edge rule removes (Sec. 2.2), and the exact
    whole-cell shift of a translated sphere only holds without such events."""
    rng = np.random.default_rng(seed)
    for _ in range(10000):
        c = tuple(float(v) for v in rng.uniform(0.3, 0.7, size=3))
        if grazing_free(np.array(c) * n, radius * n, n, cfl):
            break
    else:
        raise RuntimeError("no grazing-free centre found")
    sp = [Sphere(c, radius)]
    n3 = (n, n, n)
    phi, faces = sphere_phi_nodes_faces(n3, sp)
    s_ex = sphere_edge_roots(n3, sp) if exact else None
    return Workload("translation", n3, phi, faces, uniform_velocity(n3), cfl, steps,
                    s_exact=s_ex, shapes=sp)


def fourier_spheres(n=128, seed=2, count=8, rmin=0.05, rmax=0.12, cfl=0.5, period=2.0,
                    steps=None):
    """``count`` non-overlapping spheres in a seeded 12-mode divergence-free field
    times cos(pi t / T) on a periodic n^3 grid."""
    rng = np.random.default_rng(seed)
    sp = random_spheres(rng, count, rmin, rmax, n)
    n3 = (n, n, n)
    phi, faces = sphere_phi_nodes_faces(n3, sp)
    u = fourier_velocity(n3, rng)
    if steps is None:
        steps = int(round(period / (cfl / n)))
    return Workload("fourier_spheres", n3, phi, faces, u, cfl, steps, period=period, shapes=sp)


def batched_sizes(seed=4, count=64, sizes=(32, 48, 64, 96, 128)):
    """The seeded grid sizes of the batched instances (the first draw of
    batched_instances' generator)."""
    return [int(n) for n in np.random.default_rng(seed).choice(np.asarray(sizes), size=count)]


def batched_instances(seed=4, count=64, sizes=(32, 48, 64, 96, 128), cfl=0.5, rmin=0.07, rmax=0.15, limit=None):
    """Independent periodic instances for the batched sweeps: seeded grid sizes
    from ``sizes``, each with its own seeded 12-mode Fourier field and 1-4
    non-overlapping spheres (radii U[rmin, rmax]), dt = cfl * h of the instance.
    Returns a list of (n, phi, phi_faces, u, dt); with ``limit``, only the first
    ``limit`` instances (the same as in the full list)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    out = []
    for n in ns[:limit]:
        n = int(n)
        k = int(rng.integers(1, 5))
        sp = random_spheres(rng, k, rmin, rmax, n)
        phi, faces = sphere_phi_nodes_faces((n, n, n), sp)
        u = fourier_velocity((n, n, n), rng)
        out.append((n, phi, faces, u, cfl / n))
    return out


def cellular_velocity(n3, centre, amp=1.0, k=2):
    """Converging cellular mode about ``centre`` (x', y' = x - c_x, y - c_y, k
    cells per unit length): u_x = -amp sin(2 pi k x') cos(2 pi k y'),
    u_y = amp cos(2 pi k x') sin(2 pi k y'), u_z = 0, as the discrete curl of the
    stream function psi = -(amp / 2 pi k) sin(2 pi k x') sin(2 pi k y') sampled on
    the z-edges, so the discrete divergence vanishes.  Material on the x axis
    approaches the centre with strain rate 2 pi k amp.  Shape (3, nz, ny, nx)."""
    nx, ny, nz = n3
    x, y, _ = _grid(n3)
    w = 2 * np.pi * k
    psi = -(amp / w) * np.sin(w * (x[None, :] - centre[0])) * np.sin(w * (y[:, None] - centre[1]))
    Az = np.broadcast_to(psi[None, :, :], (nz, ny, nx))
    hx, hy = 1.0 / nx, 1.0 / ny
    ux = (np.roll(Az, -1, axis=1) - Az) / hy
    uy = -(np.roll(Az, -1, axis=2) - Az) / hx
    return np.stack([ux, uy, np.zeros((nz, ny, nx))])


def _extent(e, axis):
    """Half-width of an ellipsoid along a coordinate axis (support function)."""
    r = np.asarray(e.rot)[axis, :]
    return float(np.sqrt(np.sum((np.asarray(e.axes) * r) ** 2)))


def merging_drops(n=512, seed=5, amin_cells=40.0, amax_cells=80.0, gap_cells=8.0, fourier_scale=0.1, amp=1.0,
                  cfl=0.5, steps=200):
    """Two seeded ellipsoidal drops (semi-axes U[amin, amax] cells, random
    rotations) on the x axis through the domain centre, their supporting planes
    ``gap_cells`` apart, in a seeded 12-mode Fourier field (scaled to max
    |u| = fourier_scale) plus a converging cellular mode (amplitude ``amp``, two
    cells per unit length) centred between them, dt = cfl * h.  Exact edge
    crossings of the quadratic level sets are included.  In a divergence-free
    field the gap between the drops closes exponentially at the strain rate of
    the mode (4 pi amp), so 8 cells close to one in about ln 8 / (4 pi) time
    units (170 steps at 512^3), and the drops merge."""
    from .curvature_data import ellipsoid_fields  # local: that module builds on this one

    rng = np.random.default_rng(seed)
    h = 1.0 / n
    e1 = Ellipsoid((0.0, 0.5, 0.5), tuple(rng.uniform(amin_cells, amax_cells, 3) * h), random_rotation(rng))
    e2 = Ellipsoid((0.0, 0.5, 0.5), tuple(rng.uniform(amin_cells, amax_cells, 3) * h), random_rotation(rng))
    w1, w2 = _extent(e1, 0), _extent(e2, 0)
    d = w1 + w2 + gap_cells * h
    mid = 0.5 + float(rng.uniform(-0.5, 0.5)) * h  # off the grid lines
    e1 = Ellipsoid((mid - d / 2 - (w1 - w2) / 2, 0.5, 0.5), e1.axes, e1.rot)
    e2 = Ellipsoid((mid + d / 2 - (w1 - w2) / 2, 0.5, 0.5), e2.axes, e2.rot)
    n3 = (n, n, n)
    f = ellipsoid_fields(n3, [e1, e2])
    fin = lambda a: np.where(np.isfinite(a), a, np.sign(a))
    # the gap centre: right end of drop 1
    cx = e1.centre[0] + w1 + 0.5 * gap_cells * h
    u = fourier_scale * fourier_velocity(n3, rng) + cellular_velocity(n3, (cx, 0.5), amp)
    return Workload("merging_drops", n3, fin(f.phi), fin(f.phi_faces), u, cfl, steps, s_exact=f.s_exact,
                    shapes=[e1, e2])
