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


def test_bf16_round_matches_torch_bfloat16():
    """bf16_round against the bfloat16 conversion of torch (round to nearest,
    ties to even) on random floats over many magnitudes and on exact ties."""
    import torch

    rng = np.random.default_rng(21)
    x = (rng.normal(size=20000) * 10.0 ** rng.uniform(-8, 8, size=20000)).astype(np.float32)
    # exact ties: low 16 bits 0x8000, with even and odd bit 16
    u = rng.integers(0x3F000000, 0x47000000, size=4000, dtype=np.uint64).astype(np.uint32)
    ties = ((u & 0xFFFF0000) | 0x8000).view(np.float32)
    for v in (x, ties, -ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
        assert np.array_equal(mlp.bf16_round(v), ref)


def _net(units):
    """Parameters of a network given as a few non-zero entries:
    units = dict(W1={(j, i): w}, b1={j: b}, W2={(k, j): w}, b2={k: b}, w3={k: w}, b3=b)."""
    W1 = np.zeros((mlp.H, mlp.D_IN))
    b1, W2, b2, w3 = np.zeros(mlp.H), np.zeros((mlp.H, mlp.H)), np.zeros(mlp.H), np.zeros(mlp.H)
    for (j, i), v in units.get("W1", {}).items():
        W1[j, i] = v
    for j, v in units.get("b1", {}).items():
        b1[j] = v
    for (k, j), v in units.get("W2", {}).items():
        W2[k, j] = v
    for k, v in units.get("b2", {}).items():
        b2[k] = v
    for k, v in units.get("w3", {}).items():
        w3[k] = v
    return mlp.pack(W1, b1, W2, b2, w3, np.array([units.get("b3", 0.0)]))


def test_forward_of_closed_form_networks():
    """Networks built to compute known functions of two inputs (all values
    exact in bfloat16, so the emulated roundings change nothing): |x0 - x1|,
    max(x0, x1) for x1 >= 0, a shifted ramp with biases, a layer-2 weight off
    the diagonal (a transposed W2 gives another function), and an input in the
    tail half of the vector."""
    rng = np.random.default_rng(22)
    B = 257
    X = np.zeros((B, mlp.D_IN))
    x0 = rng.integers(-64, 65, B) / 64.0
    x1 = rng.integers(0, 65, B) / 64.0
    X[:, 3], X[:, 40] = x0, x1
    nets = [
        # |x0 - x1| = relu(x0 - x1) + relu(x1 - x0)
        (dict(W1={(0, 3): 1.0, (0, 40): -1.0, (1, 3): -1.0, (1, 40): 1.0}, W2={(0, 0): 1.0, (1, 1): 1.0},
              w3={0: 1.0, 1: 1.0}), np.abs(x0 - x1)),
        # max(x0, x1) = relu(x0 - x1) + relu(x1), x1 >= 0
        (dict(W1={(5, 3): 1.0, (5, 40): -1.0, (9, 40): 1.0}, W2={(2, 5): 1.0, (7, 9): 1.0}, w3={2: 1.0, 7: 1.0}),
         np.maximum(x0, x1)),
        # relu(x0 - 1/2) + 1/4 with the shift in b1 and b3; b2 of an idle unit is cut by its ReLU
        (dict(W1={(0, 3): 1.0}, b1={0: -0.5}, W2={(0, 0): 1.0}, b2={3: -2.0}, w3={0: 1.0, 3: 5.0}, b3=0.25),
         np.maximum(x0 - 0.5, 0.0) + 0.25),
        # 2 relu(x1) read through W2[1][0] (row: layer-2 unit, column: layer-1 unit) and b2
        (dict(W1={(0, 40): 1.0}, W2={(1, 0): 2.0}, b2={1: 0.125}, w3={1: 1.0}), 2.0 * x1 + 0.125),
    ]
    for units, ref in nets:
        p = _net(units)
        for emulate in (True, False):
            y, _ = mlp.forward(p, X, emulate=emulate)
            assert np.array_equal(y, ref), units


def test_forward_emulation_rounds_weights_and_layer1_only():
    """With emulation the layer-1 and layer-2 weights and the layer-1 activation
    are rounded to bfloat16 (8 significant bits: 1 + 2^-9 rounds to 1), the
    biases, the output weights and the layer-2 activation are not."""
    X = np.zeros((1, mlp.D_IN))
    X[0, 0] = 1.0
    e = 2.0 ** -9
    cases = [
        # a layer-1 weight 1 + e: rounded to 1
        (dict(W1={(0, 0): 1.0 + e}, W2={(0, 0): 1.0}, w3={0: 1.0}), 1.0, 1.0 + e),
        # layer-1 activation 1 + e from its bias: rounded to 1 before layer 2
        (dict(W1={(0, 0): 1.0}, b1={0: e}, W2={(0, 0): 1.0}, w3={0: 1.0}), 1.0, 1.0 + e),
        # layer-2 bias and output weight keep their bits
        (dict(W1={(0, 0): 1.0}, W2={(0, 0): 1.0}, b2={0: e}, w3={0: 1.0 + e}), (1.0 + e) ** 2, (1.0 + e) ** 2),
    ]
    for units, want_emu, want_exact in cases:
        p = _net(units)
        assert mlp.forward(p, X, emulate=True)[0][0] == want_emu
        assert mlp.forward(p, X, emulate=False)[0][0] == want_exact
