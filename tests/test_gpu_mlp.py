"""Learned curvature on the GPU (bf16 tensor-core kernels, through the C ABI) against the
FP64 oracle of oracle/mlp.py: canonical stencils bit-exact, forward pass and
gradients within the stated tolerances (bf16 operands, FP32 accumulation)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sphere_fractions(n=48, seed=3, count=3):
    w = W.fourier_spheres(n=n, seed=seed, count=count, rmin=0.08, rmax=0.2, steps=1)
    st = oracle.init(w.phi, w.phi_faces)
    C, _ = oracle.front2vof(st)
    cells = np.nonzero(((C > 0) & (C < 1)).ravel())[0].astype(np.int32)
    return w.n3, C, cells


def bf16_bits_to_f64(X):
    return X.float().cpu().numpy().astype(np.float64)


def with_satellites(C, rng, frac=0.004):
    """C plus isolated small fractions in empty cells: stencils with phase-1
    fragments (and lone interface cells)."""
    C = C.copy()
    flat = C.reshape(-1)
    empty = np.nonzero(flat == 0.0)[0]
    pick = rng.choice(empty, size=int(frac * flat.size), replace=False)
    flat[pick] = rng.uniform(0.05, 0.6, size=len(pick))
    return C


def test_gather_matches_oracle_canonical_encoding():
    n3, C, cells = sphere_fractions()
    C = with_satellites(C, np.random.default_rng(4))
    cells = np.nonzero(((C > 0) & (C < 1)).ravel())[0].astype(np.int32)
    m = ebit.Mlp()
    X, fr = m.gather(dev(C), n3, dev(cells), with_frag=True)
    blk = omlp.gather_stencils(C, cells)
    ref = omlp.encode(omlp.canonical_stencil(blk))
    assert np.array_equal(bf16_bits_to_f64(X), ref)
    fref = np.array([omlp.fragmented(b) for b in blk])
    assert fref.any() and not fref.all()
    assert np.array_equal(fr.cpu().numpy().astype(bool), fref)
    m.close()


def _random_inputs(n, rng):
    blk = rng.uniform(0, 1, size=(n, 3, 3, 3))
    return omlp.encode(omlp.canonical_stencil(blk))


PATHS = [ebit.EBIT_MLP_PATH_MMA, ebit.EBIT_MLP_PATH_TCGEN05]


@pytest.mark.parametrize("path", PATHS)
def test_forward_matches_oracle(path):
    rng = np.random.default_rng(1)
    p = omlp.init_params(2) + rng.normal(scale=0.02, size=omlp.N_PARAMS)
    p = p.astype(np.float32).astype(np.float64)
    X = _random_inputs(1000, rng)  # ragged tail: 1000 = 7 tiles of 128 + 104
    m = ebit.Mlp(p)
    m.set_path(path)
    y = m.forward(dev(X).to(torch.bfloat16)).cpu().numpy()
    m.sync()
    yr, _ = omlp.forward(p, X, emulate=True)
    err = np.abs(y - yr)
    assert np.max(err / (np.abs(yr) + 0.1)) <= 2e-3, np.max(err)
    m.close()


def test_gradient_matches_oracle_backprop():
    rng = np.random.default_rng(5)
    p = omlp.init_params(4) + rng.normal(scale=0.02, size=omlp.N_PARAMS)
    p = p.astype(np.float32).astype(np.float64)
    B = 640
    X = _random_inputs(B, rng)
    t = rng.uniform(0.05, 0.8, size=B).astype(np.float32).astype(np.float64)
    m = ebit.Mlp(p)
    g = m.gradient(dev(X).to(torch.bfloat16), dev(t.astype(np.float32))).cpu().numpy().astype(np.float64)
    m.sync()
    _, gr = omlp.loss_and_grad(p, X, t, emulate=True)
    blocks = [("W1", 0, 128 * 64), ("b1", 8192, 8320), ("W2", 8320, 8320 + 16384), ("b2", 24704, 24832),
              ("w3", 24832, 24960), ("b3", 24960, 24961)]
    # element by element: |g - g_ref| <= 1e-2 |g_ref| + 1e-3 max|g_ref| in each
    # block (the kernel rounds the backward operands to bf16 for the tensor
    # cores; the oracle passes the roundings straight through)
    for name, a, b in blocks:
        err = np.abs(g[a:b] - gr[a:b])
        bound = 1e-2 * np.abs(gr[a:b]) + 1e-3 * np.abs(gr[a:b]).max()
        assert np.all(err <= bound), (name, int(np.sum(err > bound)), float(np.max(err / bound)))
    m.close()


def test_training_steps_reduce_the_loss():
    rng = np.random.default_rng(9)
    X = _random_inputs(4096, rng)
    # a smooth target of the stencil: a fixed random linear map of the heads
    wv = rng.normal(size=27)
    t = (0.3 + 0.05 * np.tanh(X[:, :27] @ wv)).astype(np.float32)
    m = ebit.Mlp(omlp.init_params(0))
    Xd, td = dev(X).to(torch.bfloat16), dev(t)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.train_step(Xd, td, 1e-3, loss)
    first = loss.item()
    for _ in range(300):
        m.train_step(Xd, td, 1e-3, loss)
    m.sync()
    assert loss.item() < 0.2 * first, (first, loss.item())
    m.close()


def test_indexed_training_step_equals_the_gathered_batch():
    rng = np.random.default_rng(13)
    X = _random_inputs(3000, rng)
    t = rng.uniform(0.05, 0.6, size=3000).astype(np.float32)
    idx = rng.permutation(3000)[:1000].astype(np.int32)
    p0 = omlp.init_params(5)
    a, b = ebit.Mlp(p0), ebit.Mlp(p0)
    Xd, td = dev(X).to(torch.bfloat16), dev(t)
    la = torch.zeros(1, dtype=torch.float32, device="cuda")
    lb = torch.zeros(1, dtype=torch.float32, device="cuda")
    a.train_step(Xd, td, 1e-3, la, idx=dev(idx), batch=1000)
    b.train_step(Xd[dev(idx).long()].contiguous(), td[dev(idx).long()].contiguous(), 1e-3, lb)
    a.sync()
    b.sync()
    pa, pb = a.get_params().cpu().numpy(), b.get_params().cpu().numpy()
    # the same step up to the order of the FP32 gradient sums
    assert np.max(np.abs(pa - pb)) <= 1e-6, np.max(np.abs(pa - pb))
    assert abs(la.item() - lb.item()) <= 1e-4 * abs(lb.item())
    a.close()
    b.close()


@pytest.mark.parametrize("path", PATHS)
def test_curvature_mode_with_height_function_fallback_matches_oracle(path):
    n3, C, _ = sphere_fractions()
    C = with_satellites(C, np.random.default_rng(6))
    rng = np.random.default_rng(8)
    p = omlp.init_params(7) + rng.normal(scale=0.01, size=omlp.N_PARAMS)
    p = p.astype(np.float32).astype(np.float64)
    hf_kh, hf_st = oracle.hf_curvature(C)
    # shift the output bias so that about half the cells leave |kappa h| <= 1
    _, _, _, y0, _ = omlp.learned_curvature(C, p, 1, hf_kh, hf_st)
    p[-1] += 1.0 - np.median(y0)
    p = p.astype(np.float32).astype(np.float64)
    cells, kh_ref, st_ref, y_ref, frag = omlp.learned_curvature(C, p, 2, hf_kh, hf_st)
    assert frag.any() and (np.abs(y_ref) > 1.0).any() and (np.abs(y_ref) <= 1.0).any()
    m = ebit.Mlp(p)
    m.set_path(path)
    g = ebit.Grid(*n3)
    g.set_mlp(m)
    Cd = dev(C)
    kh = torch.zeros_like(Cd)
    st = torch.zeros(Cd.shape, dtype=torch.uint8, device="cuda")
    g.curvature(Cd, kh, st, mode=ebit.EBIT_CURV_MLP_HF, flags=ebit.EBIT_FULL)
    g.sync()
    kh_h = kh.cpu().numpy().ravel()
    st_h = st.cpu().numpy().ravel()
    assert np.array_equal(np.nonzero(st_h)[0], np.sort(cells))
    clear = np.abs(np.abs(y_ref) - 1.0) > 1e-2   # the FP32 and FP64 decisions agree away from 1
    assert np.array_equal(st_h[cells][clear], st_ref[clear])
    hf = clear & (st_ref != 5)
    assert np.all(np.abs(kh_h[cells][hf] - kh_ref[hf]) <= 1e-12)
    learned = clear & (st_ref == 5)
    assert np.max(np.abs(kh_h[cells][learned] - y_ref[learned]) / (np.abs(y_ref[learned]) + 0.1)) <= 2e-3
    g.close()
    m.close()


def test_curvature_mode_uses_the_network():
    n3, C, cells = sphere_fractions()
    rng = np.random.default_rng(2)
    p = omlp.init_params(7) + rng.normal(scale=0.01, size=omlp.N_PARAMS)
    m = ebit.Mlp(p)
    g = ebit.Grid(*n3)
    g.set_mlp(m)
    Cd = dev(C)
    kh = torch.zeros_like(Cd)
    st = torch.zeros(Cd.shape, dtype=torch.uint8, device="cuda")
    g.curvature(Cd, kh, st, mode=ebit.EBIT_CURV_MLP, flags=ebit.EBIT_FULL)
    X = m.gather(Cd, n3, dev(cells))
    y = m.forward(X).cpu().numpy()
    st_h = st.cpu().numpy().ravel()
    assert np.all(st_h[cells] == ebit.ST_MLP)
    assert np.array_equal(np.nonzero(st_h)[0], np.sort(cells))
    assert np.allclose(kh.cpu().numpy().ravel()[cells], y, rtol=0, atol=1e-6)
    g.close()
    m.close()


def test_context_owned_network_equals_attached_network():
    n3, C, cells = sphere_fractions()
    p = omlp.init_params(3).astype(np.float32)
    m = ebit.Mlp(p.astype(np.float64))
    g1, g2 = ebit.Grid(*n3), ebit.Grid(*n3)
    g1.set_mlp(m)
    g2.load_mlp(p)
    Cd = dev(C)
    outs = []
    for g in (g1, g2):
        kh = torch.zeros_like(Cd)
        st = torch.zeros(Cd.shape, dtype=torch.uint8, device="cuda")
        g.curvature(Cd, kh, st, mode=ebit.EBIT_CURV_MLP, flags=ebit.EBIT_FULL)
        outs.append((kh, st))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    short = torch.zeros(5, dtype=torch.float32)
    assert ebit.load().ebit_mlp_load(g2.ctx, ctypes.c_void_p(short.data_ptr()), 20) == ebit.EBIT_EINVAL
    g1.close()
    g2.close()
    m.close()


def test_tensor_paths_agree_on_the_curvature_field():
    n3, C, cells = sphere_fractions()
    C = with_satellites(C, np.random.default_rng(11))
    p = omlp.init_params(9) + np.random.default_rng(3).normal(scale=0.01, size=omlp.N_PARAMS)
    m = ebit.Mlp(p)
    g = ebit.Grid(*n3)
    g.set_mlp(m)
    Cd = dev(C)
    out = []
    for path in PATHS:
        m.set_path(path)
        kh = torch.zeros_like(Cd)
        st = torch.zeros(Cd.shape, dtype=torch.uint8, device="cuda")
        g.curvature(Cd, kh, st, mode=ebit.EBIT_CURV_MLP, flags=ebit.EBIT_FULL)
        assert m.sync() == 0
        out.append((kh.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][1], out[1][1])
    # the same bf16 products, FP32 sums in a different order
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-5
    g.close()
    m.close()


def test_training_step_is_the_gradient_then_adam_and_reports_each_batch_loss():
    """One training step equals the library's gradient followed by Adam written
    out on the host (FP32, the kernel's order of operations), and each step
    reports the loss of its own batch at the parameters it started from: the
    device-pointer and host-pointer paths, two steps in a row (the loss is
    cleared between steps)."""
    rng = np.random.default_rng(21)
    p0 = (omlp.init_params(6) + rng.normal(scale=0.02, size=omlp.N_PARAMS)).astype(np.float32)
    B, lr = 640, 1e-3
    X = _random_inputs(B, rng)
    t = rng.uniform(0.05, 0.8, size=B).astype(np.float32)
    Xd, td = dev(X).to(torch.bfloat16), dev(t)
    m = ebit.Mlp(p0.astype(np.float64))
    g = m.gradient(Xd, td).cpu().numpy().astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.train_step(Xd, td, lr, loss)
    m.sync()
    p1 = m.get_params().cpu().numpy().astype(np.float32)
    # Adam step 1 in float32 (m0 = v0 = 0)
    b1, b2, eps = np.float32(0.9), np.float32(0.999), np.float32(1e-8)
    mh = np.float32(1.0 - b1) * g
    vh = np.float32(1.0 - b2) * g * g
    bc1, bc2 = np.float32(1.0) - b1, np.float32(1.0) - b2
    ph = p0 - np.float32(lr) * (mh / bc1) / (np.sqrt(vh / bc2) + eps)
    # where the gradient is not tiny the step does not depend on the order of
    # the FP32 gradient sums of the two launches; elsewhere it is at most lr
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert big.sum() > 0.3 * big.size
    assert np.max(np.abs(p1 - ph)[big]) <= 1e-6, np.max(np.abs(p1 - ph)[big])
    assert np.max(np.abs(p1 - p0)) <= 1.001 * lr
    Xh = bf16_bits_to_f64(Xd)
    l0, _ = omlp.loss_and_grad(p0.astype(np.float64), Xh, t.astype(np.float64), emulate=True)
    assert abs(loss.item() / B - l0) <= 2e-2 * l0, (loss.item() / B, l0)
    # second step, loss into host memory through the C ABI
    cf = ctypes.c_float(-1.0)
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    rc = ebit.load().ebit_mlp_train_step(m.h, P(Xd), P(td), None, B, ctypes.c_float(lr),
                                          ctypes.c_void_p(ctypes.addressof(cf)))
    assert rc == 0
    m.sync()
    l1, _ = omlp.loss_and_grad(p1.astype(np.float64), Xh, t.astype(np.float64), emulate=True)
    assert abs(cf.value / B - l1) <= 2e-2 * l1, (cf.value / B, l1, l0)
    m.close()
