"""Pins of the oracle's three-dimensional height-function curvature (the HF
method that Sec. 2.6 uses for the surface-tension term) against closed forms:

* spheres of radius 8, 16 and 32 cells, both phases: kappa*h -> +-2h/R with
  about second-order decrease (the sum of two equal principal curvatures);
* an axis-aligned ellipsoid: kappa*h against the mean curvature of the quadric
  at the surface point on each cell's height-function column (heights with a
  non-zero cross derivative h_xy and unequal slopes h_x != h_y);
* a cylinder whose axis (1, 2, 0) is not aligned with the grid: kappa*h = h/R
  (one principal curvature, cross derivative non-zero).

A wrong weight on the h_xy term, a flipped sign of the cross term or swapped
(1 + h_x^2), (1 + h_y^2) weights fails these pins; the z-cylinder and plane
pins cannot see any of them (there h_xy = 0 and one slope vanishes).

Volume fractions are computed here, independently of the oracle's Front2VOF:
each cut cell's volume is a one-dimensional Gauss-Legendre quadrature over
slices whose area has a closed form (disk or strip inside a rectangle), split
where the slice's shape changes so that every piece is smooth.  The quadrature
itself is checked against the closed-form total volume of each body.
"""
import numpy as np
import pytest

import oracle

GL_T, GL_W = np.polynomial.legendre.leggauss(16)
GL_T = 0.5 * (GL_T + 1.0)  # nodes and weights on [0, 1]
GL_W = 0.5 * GL_W


# ------------------------------------------------------------ slice areas
def disk_rect_area(r, yc, zc, y0, y1, z0, z1):
    """Area of the disk of radius r centred (yc, zc) inside [y0,y1] x [z0,z1].

    The z-extent of the disk above a point y is [zc - w, zc + w] with
    w = sqrt(r^2 - (y - yc)^2); the area is the integral over y of that extent
    clipped to [z0, z1].  The clipped extent changes form only where w equals
    |z0 - zc| or |z1 - zc| or vanishes, so between those points it is z1 - z0,
    zc + w - z0, z1 - zc + w, 2w or 0, each integrated exactly with the
    antiderivative of w.  All arguments broadcast."""
    r, yc, zc, y0, y1, z0, z1 = np.broadcast_arrays(*(np.asarray(v, np.float64) for v in (r, yc, zc, y0, y1, z0, z1)))
    # work in u = y - yc so that the ends u = +-r of the chord are exact
    u0, u1 = y0 - yc, y1 - yc
    cand = [u0, u1, -r, r]
    for d in (z0 - zc, z1 - zc):
        t = np.sqrt(np.maximum(r * r - d * d, 0.0))
        cand += [-t, t]
    P = np.sort(np.clip(np.stack(cand, -1), u0[..., None], u1[..., None]), axis=-1)
    rs = np.where(r > 0, r, 1.0)

    def W(u):  # antiderivative of w(u) = sqrt(r^2 - u^2) on |u| <= r
        u = np.clip(u, -r, r)
        w = np.sqrt(np.maximum(r * r - u * u, 0.0))
        return 0.5 * (u * w + r * r * np.arcsin(np.clip(u / rs, -1.0, 1.0)))

    tot = np.zeros(r.shape)
    for k in range(P.shape[-1] - 1):
        a, b = P[..., k], P[..., k + 1]
        um = 0.5 * (a + b)
        wm = np.sqrt(np.maximum(r * r - um * um, 0.0))
        live = (np.abs(um) < r) & (np.minimum(z1, zc + wm) > np.maximum(z0, zc - wm)) & (b > a)
        L = b - a
        Wd = W(b) - W(a)
        upper = np.where(zc + wm >= z1, z1 * L, zc * L + Wd)
        lower = np.where(zc - wm <= z0, z0 * L, zc * L - Wd)
        tot += np.where(live, upper - lower, 0.0)
    return tot


def halfplane_rect_area(al, be, c, x0, y0):
    """Area of {al x + be y <= c} inside the unit square [x0,x0+1] x [y0,y0+1]
    (al, be != 0): the two-dimensional form of the half-space volume,
    sum over corners v of (-1)^{|v|} max(0, c - n.v)^2 / (2 al be) after
    reflecting so that al, be > 0."""
    c = c - al * x0 - be * y0
    if al < 0:
        c, al = c - al, -al
    if be < 0:
        c, be = c - be, -be
    tot = 0.0
    for vx in (0, 1):
        for vy in (0, 1):
            tot = tot + (-1) ** (vx + vy) * np.maximum(0.0, c - al * vx - be * vy) ** 2
    return np.clip(tot / (2.0 * al * be), 0.0, 1.0)


def integrate_pieces(f, lo, hi, breaks):
    """Integral of f over [lo, hi] (arrays over cells), split at the given break
    points (cells x m array, NaN for none).  Each piece [a, b] is mapped by
    z = a + (b - a)(3t^2 - 2t^3), which removes the square-root endpoint
    behaviour of a slice area, then integrated by 16-point Gauss-Legendre."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    br = np.where(np.isnan(breaks), lo[:, None], breaks)
    P = np.sort(np.clip(np.concatenate([lo[:, None], hi[:, None], br], 1), lo[:, None], hi[:, None]), axis=1)
    a, b = P[:, :-1, None], P[:, 1:, None]
    t = GL_T[None, None, :]
    s = t * t * (3.0 - 2.0 * t)
    ds = 6.0 * t * (1.0 - t)
    z = a + (b - a) * s
    vals = f(z)
    return np.sum(vals * (b - a) * ds * GL_W[None, None, :], axis=(1, 2))


# -------------------------------------------------------- volume fractions
def ellipsoid_fractions(n3, centre, axes, chunk=4000):
    """Volume fractions of the axis-aligned ellipsoid sum ((x_i - c_i)/a_i)^2 <= 1
    on an (nz, ny, nx) grid of unit cells (cell (i,j,k) = [i,i+1]x[j,j+1]x[k,k+1]).
    Slices at fixed x are ellipses; scaling z by b/c makes them disks."""
    nx, ny, nz = n3
    cx, cy, cz = centre
    a, b, c = axes
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    corners = [((i + dx - cx) / a) ** 2 + ((j + dy - cy) / b) ** 2 + ((k + dz - cz) / c) ** 2
               for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]
    inside = np.all([q <= 1.0 for q in corners], axis=0)  # convex body: all corners in
    near = [np.maximum(np.maximum(lo - cc, 0.0), cc - (lo + 1)) / ax for lo, cc, ax in ((i, cx, a), (j, cy, b), (k, cz, c))]
    outside = near[0] ** 2 + near[1] ** 2 + near[2] ** 2 >= 1.0  # nearest point of the scaled box
    C = np.where(inside, 1.0, 0.0)
    cut = np.argwhere(~inside & ~outside)
    sc = b / c
    for p in range(0, len(cut), chunk):
        kk, jj, ii = (cut[p:p + chunk, q].astype(np.float64) for q in range(3))
        y0, y1, z0, z1 = jj, jj + 1, kk * sc, (kk + 1) * sc
        zc = cz * sc
        ds = [np.abs(y0 - cy), np.abs(y1 - cy), np.abs(z0 - zc), np.abs(z1 - zc)]
        ds += [np.hypot(yy - cy, zz - zc) for yy in (y0, y1) for zz in (z0, z1)]
        br = []
        for d in ds + [np.zeros_like(y0)]:
            e = 1.0 - (d / b) ** 2
            t = np.where(e > 0, a * np.sqrt(np.maximum(e, 0.0)), np.nan)
            br += [cx - t, cx + t]
        br = np.stack(br, 1)

        def area(x, y0=y0, y1=y1, z0=z0, z1=z1, zc=zc):
            q2 = 1.0 - ((x - cx) / a) ** 2
            r = b * np.sqrt(np.maximum(q2, 0.0))
            ex = lambda v: v[:, None, None]
            return disk_rect_area(r, cy, zc, ex(y0), ex(y1), ex(z0), ex(z1)) / sc

        C[kk.astype(int), jj.astype(int), ii.astype(int)] = integrate_pieces(area, ii, ii + 1, br)
    return C


def oblique_cylinder_fractions(n, nz, point, R, chunk=4000):
    """Volume fractions of the periodic cylinder of radius R whose axis runs
    along (1, 2, 0)/sqrt(5) through ``point``, on an (nz, n, n) grid periodic in
    x and y.  Slices at fixed z are strips |u| <= sqrt(R^2 - (z - pz)^2) with
    u = (2 (x - px) - (y - py)) / sqrt(5) the signed distance from the axis in
    the xy plane; the copies of the axis shifted by the periodic lattice lie
    n/sqrt(5) apart in u.  Returns C and the period of u."""
    px, py, pz = point
    al, be = 2.0 / np.sqrt(5.0), -1.0 / np.sqrt(5.0)  # u = al (x - px) + be (y - py)
    period = n / np.sqrt(5.0)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    u = al * (i + 0.5 - px) + be * (j + 0.5 - py)
    shift = period * np.round(u / period)
    ur = u - shift
    dist = np.hypot(ur, k + 0.5 - pz)
    C = np.where(dist < R, 1.0, 0.0)
    cut = np.argwhere(np.abs(dist - R) < 1.0)  # the cell's half-diagonal is 0.87
    for p in range(0, len(cut), chunk):
        kk, jj, ii = (cut[p:p + chunk, q] for q in range(3))
        sh = shift[kk, jj, ii]
        x0, y0 = ii.astype(np.float64), jj.astype(np.float64)
        c0 = al * px + be * py + sh  # u = al x + be y - c0
        uc = [al * (x0 + dx) + be * (y0 + dy) - c0 for dx in (0, 1) for dy in (0, 1)]
        br = []
        for uu in uc + [np.zeros_like(x0)]:
            e = R * R - uu * uu
            t = np.where(e > 0, np.sqrt(np.maximum(e, 0.0)), np.nan)
            br += [pz - t, pz + t]
        br = np.stack(br, 1)

        def area(z, x0=x0, y0=y0, c0=c0):
            w = np.sqrt(np.maximum(R * R - (z - pz) ** 2, 0.0))
            ex = lambda v: v[:, None, None]
            hi = halfplane_rect_area(al, be, ex(c0) + w, ex(x0), ex(y0))
            lo = halfplane_rect_area(al, be, ex(c0) - w, ex(x0), ex(y0))
            return hi - lo

        C[kk, jj, ii] = integrate_pieces(area, kk.astype(np.float64), kk + 1.0, br)
    return C, period


# ------------------------------------------------ analytic mean curvature
def ellipsoid_kappa(p, centre, axes):
    """Mean curvature (sum of principal curvatures) of F = sum (x_i/a_i)^2 - 1 at
    p: (|grad F|^2 tr H - grad F^T H grad F) / |grad F|^3, positive for the
    body's own phase (2/R on a sphere)."""
    g = np.array([2.0 * (p[q] - centre[q]) / axes[q] ** 2 for q in range(3)])
    Hd = np.array([2.0 / axes[q] ** 2 for q in range(3)])
    g2 = np.sum(g * g, axis=0)
    return (g2 * Hd.sum() - np.sum(Hd[:, None] * g * g, axis=0)) / g2 ** 1.5


def column_points(cells, status, centre, axes):
    """Surface point on each cell's height-function column: the line through the
    cell centre along the axis named by the status, root nearest the centre."""
    pts = (cells[:, ::-1] + 0.5).T.astype(np.float64)  # x, y, z rows
    d = status.astype(int) - 1
    out = pts.copy()
    for ax in range(3):
        m = d == ax
        rest = sum(((pts[q][m] - centre[q]) / axes[q]) ** 2 for q in range(3) if q != ax)
        e = np.sqrt(np.maximum(1.0 - rest, 0.0)) * axes[ax]
        r1, r2 = centre[ax] + e, centre[ax] - e
        out[ax][m] = np.where(np.abs(r1 - pts[ax][m]) < np.abs(r2 - pts[ax][m]), r1, r2)
    return out


# ------------------------------------------------------------------- pins
def test_quadrature_volumes_match_closed_forms():
    """The test's own volume fractions: totals equal the closed-form volumes."""
    n = 40
    cen, ax = (19.3, 20.6, 18.9), (9.5, 12.25, 14.75)
    C = ellipsoid_fractions((n, n, n), cen, ax)
    assert C.min() >= 0.0 and C.max() <= 1.0
    assert abs(C.sum() - 4.0 / 3.0 * np.pi * np.prod(ax)) <= 1e-9 * C.sum()
    Cs = ellipsoid_fractions((n, n, n), cen, (11.0, 11.0, 11.0))
    assert abs(Cs.sum() - 4.0 / 3.0 * np.pi * 11.0 ** 3) <= 1e-9 * Cs.sum()
    nz, R = 24, 6.5
    Cc, period = oblique_cylinder_fractions(n, nz, (3.3, 7.1, 11.6), R)
    length = n * np.sqrt(5.0)  # the axis crosses the periodic box once in x, twice in y
    assert abs(Cc.sum() - np.pi * R * R * length) <= 1e-9 * Cc.sum()


SPHERE_RADII = (8.0, 16.0, 32.0)


@pytest.fixture(scope="module")
def sphere_errors():
    rng = np.random.default_rng(91)
    out = {}
    for R in SPHERE_RADII:
        n = int(2 * R + 14)
        cen = tuple(n / 2 + rng.uniform(-0.5, 0.5, 3))
        C = ellipsoid_fractions((n, n, n), cen, (R, R, R))
        for inside in (1, 0):
            kh, st = oracle.hf_curvature(C if inside else 1.0 - C)
            ok = (st >= 1) & (st <= 3)
            iface = st > 0
            ref = (2.0 if inside else -2.0) / R
            rel = np.abs(kh[ok] - ref) / abs(ref)
            out[(R, inside)] = (rel, ok.sum() / iface.sum())
    return out


@pytest.mark.parametrize("inside", [1, 0])
def test_hf_spheres_converge_to_two_over_r(sphere_errors, inside):
    """kappa*h of spheres of radius 8, 16, 32 cells against 2h/R (negative for the
    complement phase): small relative error, the RMS falling by about 4 per
    halving of h/R, and a valid height-function stencil at most interface cells
    (columns of 9 cells find pure ends less often on small spheres)."""
    rms, mx = [], []
    for R, cover_min in zip(SPHERE_RADII, (0.8, 0.93, 0.97)):
        rel, cover = sphere_errors[(R, inside)]
        assert cover >= cover_min, (R, cover)
        rms.append(np.sqrt(np.mean(rel ** 2)))
        mx.append(rel.max())
    assert rms[0] < 0.008 and mx[0] < 0.03, (rms, mx)
    for q in range(len(SPHERE_RADII) - 1):
        assert rms[q + 1] < rms[q] / 2.8, rms
    assert mx[2] < 0.006 and mx[2] < mx[0] / 3.0, mx


def test_hf_ellipsoid_mean_curvature():
    """Axis-aligned ellipsoid with semi-axes 11, 15 and 20 cells: kappa*h at
    every interface cell with a valid stencil against the mean curvature of the
    quadric at the surface point on that cell's height-function column."""
    n = 56
    cen, ax = (27.37, 28.11, 27.73), (11.0, 15.0, 20.0)
    C = ellipsoid_fractions((n, n, n), cen, ax)
    kh, st = oracle.hf_curvature(C)
    cells = np.argwhere((st >= 1) & (st <= 3))
    assert len(cells) >= 0.9 * (st > 0).sum()
    p = column_points(cells, st[tuple(cells.T)], cen, ax)
    ref = ellipsoid_kappa(p, cen, ax)
    got = kh[tuple(cells.T)]
    rel = np.abs(got - ref) / ref
    assert np.sqrt(np.mean(rel ** 2)) < 0.006, np.sqrt(np.mean(rel ** 2))
    assert rel.max() < 0.05, rel.max()
    # the complement phase gives the opposite curvature
    kh2, st2 = oracle.hf_curvature(1.0 - C)
    assert np.array_equal(st2, st)
    assert np.abs(kh2[tuple(cells.T)] + got).max() <= 1e-12


def test_hf_oblique_cylinder():
    """Cylinder of radius 8 cells along (1, 2, 0): kappa*h = 1/R at every interface
    cell with a valid stencil.  Its heights along z vary with both x and y (h_xy
    non-zero), and so do its heights along x (with y and z)."""
    n, nz, R = 80, 30, 8.0
    C, _ = oblique_cylinder_fractions(n, nz, (10.37, 3.71, 14.83), R)
    kh, st = oracle.hf_curvature(C)
    ok = (st >= 1) & (st <= 3)
    assert ok.sum() >= 0.88 * (st > 0).sum()
    # |n_x| = 2 |n_y| on this cylinder: columns run along x or z
    assert set(np.unique(st[ok])) == {1, 3}
    rel = np.abs(kh[ok] * R - 1.0)
    assert np.sqrt(np.mean(rel ** 2)) < 0.009, np.sqrt(np.mean(rel ** 2))
    assert rel.max() < 0.025, rel.max()
