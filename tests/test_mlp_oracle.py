"""Pins of the FP64 learned-curvature oracle (oracle/mlp.py) against
mathematics it does not share code with."""
import itertools

import numpy as np

from oracle import mlp


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3) + rng.normal(scale=0.05, size=mlp.N_PARAMS)
    X = rng.uniform(0, 1, size=(7, mlp.D_IN))
    t = rng.uniform(0.1, 0.8, size=7)
    loss, g = mlp.loss_and_grad(p, X, t, emulate=False)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2]])
    for i in idx:
        e = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        num = (mlp.loss_and_grad(pp, X, t, emulate=False)[0] - mlp.loss_and_grad(pm, X, t, emulate=False)[0]) / (2 * e)
        assert abs(num - g[i]) <= 1e-6 * max(1e-3, abs(num)) + 1e-9, (i, num, g[i])


def _symmetries():
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((1, -1), repeat=3):
            yield perm, flips


def _apply(blk, perm, flips):
    """Stencil of the same shape seen through an axis permutation and reflections."""
    out = np.zeros_like(blk)
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        d = (dx, dy, dz)
        e = [0, 0, 0]
        for a in range(3):
            e[perm[a]] = flips[a] * d[a]
        out[e[2] + 1, e[1] + 1, e[0] + 1] = blk[dz + 1, dy + 1, dx + 1]
    return out


def test_canonical_stencil_invariant_under_the_48_symmetries():
    rng = np.random.default_rng(2)
    for _ in range(20):
        # a smooth fraction field around a cell: generic normal, no ties
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        kap = rng.uniform(-0.2, 0.2)
        blk = np.zeros((3, 3, 3))
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            s = nrm[0] * dx + nrm[1] * dy + nrm[2] * dz + kap * (dx * dx + dy * dy + dz * dz) + rng.uniform(-0.3, 0.3)
            blk[dz + 1, dy + 1, dx + 1] = np.clip(0.5 - s, 0.0, 1.0)
        ref = mlp.canonical_stencil(blk)
        for perm, flips in _symmetries():
            got = mlp.canonical_stencil(_apply(blk, perm, flips))
            assert np.array_equal(got, ref)
        # canonical frame: reflected normal has 0 <= n0 <= n1 <= n2
        n = mlp.youngs_normal(ref.reshape(3, 3, 3))
        assert np.all(n >= 0) and n[0] <= n[1] <= n[2]


def test_ellipsoid_curvature_closed_forms():
    a, b, c = 3.0, 5.0, 7.0
    # pole of the x axis: principal curvatures a/b^2 and a/c^2
    k = mlp.ellipsoid_mean_curvature(np.array([a, 0.0, 0.0]), (a, b, c))
    assert abs(k - (a / b ** 2 + a / c ** 2)) <= 1e-14
    k = mlp.ellipsoid_mean_curvature(np.array([0.0, 0.0, c]), (a, b, c))
    assert abs(k - (c / a ** 2 + c / b ** 2)) <= 1e-14
    # sphere: 2/R everywhere
    rng = np.random.default_rng(4)
    x = rng.normal(size=(50, 3))
    x = 4.0 * x / np.linalg.norm(x, axis=1, keepdims=True)
    assert np.allclose(mlp.ellipsoid_mean_curvature(x, (4.0, 4.0, 4.0)), 0.5, rtol=0, atol=1e-14)


def test_ellipsoid_curvature_matches_divergence_of_the_normal():
    axes = (2.0, 3.0, 5.0)
    rng = np.random.default_rng(5)
    for _ in range(10):
        d = rng.normal(size=3)
        x0 = d / np.sqrt(np.sum(d * d / np.array(axes) ** 2))  # on the surface

        def nhat(x):
            g = 2 * x / np.array(axes) ** 2
            return g / np.linalg.norm(g)
        e = 1e-5
        div = sum((nhat(x0 + e * np.eye(3)[i])[i] - nhat(x0 - e * np.eye(3)[i])[i]) / (2 * e) for i in range(3))
        # the divergence of the extended unit normal field equals the mean-curvature sum
        assert abs(div - mlp.ellipsoid_mean_curvature(x0, axes)) <= 1e-6


def test_closest_point_is_on_the_surface_along_the_normal():
    axes = (2.0, 3.0, 5.0)
    rng = np.random.default_rng(6)
    p = rng.normal(scale=4.0, size=(200, 3))
    x = mlp.ellipsoid_closest_point(p, axes)
    assert np.allclose(np.sum(x * x / np.array(axes) ** 2, axis=1), 1.0, atol=1e-10)
    g = x / np.array(axes) ** 2
    cross = np.cross(p - x, g)
    assert np.max(np.abs(cross)) <= 1e-8


def test_first_adam_step_closed_form():
    p = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, -1e-4, 5.0])
    m = np.zeros(5)
    v = np.zeros(5)
    p1, m1, v1 = mlp.adam(p, g, m, v, 1, lr=0.01)
    # bias-corrected first step: -lr * g / (|g| + eps)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_bf16_split_reconstructs_float32():
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, size=10000)
    hi, lo = mlp.split_bf16(x)
    f = x.astype(np.float32).astype(np.float64)
    assert np.max(np.abs(hi + lo - f)) <= 2.0 ** -16 * 2 ** -1 * 1.0001
    # heads are bfloat16 values: low 16 bits of the float32 pattern are zero
    assert np.all((hi.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_fragment_rule_matches_connected_component_labelling():
    from scipy import ndimage
    rng = np.random.default_rng(11)
    st6 = ndimage.generate_binary_structure(3, 1)
    seen = {True: 0, False: 0}
    for trial in range(3000):
        dens = rng.uniform(0.15, 0.9)
        blk = np.where(rng.uniform(size=(3, 3, 3)) < dens, rng.uniform(0.01, 1.0, size=(3, 3, 3)), 0.0)
        if trial % 2 == 0:
            blk[1, 1, 1] = 0.5
        lab, _ = ndimage.label(blk > 0, structure=st6)
        if blk[1, 1, 1] > 0:
            expect = bool(np.any((blk > 0) & (lab != lab[1, 1, 1])))
        else:
            expect = bool(np.any(blk > 0))
        assert mlp.fragmented(blk) == expect
        seen[expect] += 1
    assert seen[True] > 100 and seen[False] > 100
    # a face-connected snake through the block is one piece; a diagonal neighbour is not
    snake = np.zeros((3, 3, 3))
    for z, y, x in [(1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2), (2, 2, 1), (2, 2, 0), (2, 1, 0), (2, 0, 0)]:
        snake[z, y, x] = 0.4
    assert not mlp.fragmented(snake)
    diag = np.zeros((3, 3, 3))
    diag[1, 1, 1] = diag[2, 2, 2] = 0.5
    assert mlp.fragmented(diag)


def test_learned_curvature_fallback_selection():
    rng = np.random.default_rng(12)
    C = np.zeros((8, 8, 8))
    C[3:5, 3:5, 3:5] = rng.uniform(0.2, 0.8, size=(2, 2, 2))
    C[2, 2, 2] = 0.3                      # touches the cube only along a corner
    p = mlp.init_params(1)
    hf_kh = np.full(C.size, 7.0)
    hf_st = np.full(C.size, 2, dtype=np.uint8)
    cells, kh, st, y, frag = mlp.learned_curvature(C, p, 2, hf_kh, hf_st)
    assert len(cells) == 9
    for c, k, s_, yy, f in zip(cells, kh, st, y, frag):
        if f or abs(yy) > 1.0:
            assert k == 7.0 and s_ == 2
        else:
            assert k == yy and s_ == 5
    assert frag.any() and not frag.all()
    cells1, kh1, st1, y1, _ = mlp.learned_curvature(C, p, 1, hf_kh, hf_st)
    assert np.array_equal(kh1, y1) and np.all(st1 == 5)
