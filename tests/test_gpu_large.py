"""The two large configurations: converging ellipsoidal drops that merge
(topology change through the colour field), and the 512^3 domain in the launch
configuration of the benchmark, checked against the oracle on windows.

The oracle is global and periodic, so a 512^3 grid is out of its reach; every
operation of the method is local (a sweep reads at most three cells along the
sweep axis and one across, Front2VOF one cell, height functions five), so the
oracle run on a window of the GPU state must agree with the GPU result away
from the window's seams."""
import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import learned
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def components(cb):
    lab, n = ndimage.label((cb & 1).astype(bool))
    # periodic: merge labels that touch across the domain faces
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for ax in range(3):
        a = np.take(lab, 0, axis=ax)
        b = np.take(lab, -1, axis=ax)
        m = (a > 0) & (b > 0)
        for x, y in zip(a[m], b[m]):
            parent[find(x)] = find(y)
    return len({find(k) for k in range(1, n + 1)})


def test_converging_drops_merge():
    w = W.merging_drops(n=256, seed=5, amin_cells=20.0, amax_cells=40.0, gap_cells=8.0)
    g = ebit.Grid(*w.n3)
    g.init(dev(w.phi), dev(w.phi_faces), dev(w.s_exact))
    mlp = learned.load_network()
    g.set_mlp(mlp)
    cb0, _ = g.get_state()
    assert components(cb0.cpu().numpy()) == 2
    ud = [dev(w.u[d]) for d in range(3)]
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    g.front2vof(C, ebit.EBIT_FULL)
    v0 = float(C.sum())
    merged_at = None
    for n in range(200):
        g.step(n, ud, w.lam(n) * g.h)
        g.front2vof(C)
        g.curvature(C, kh, st, mode=ebit.EBIT_CURV_MLP_HF)
        if n % 8 == 7:
            cb, _ = g.get_state()
            if components(cb.cpu().numpy()) == 1:
                merged_at = n
                break
    g.sync()
    assert merged_at is not None, "the drops did not merge"
    cnt = g.counters()
    assert cnt["annihilate"] > 0          # markers met and vanished: the colour field joined the drops
    # volume is kept to within the method's advection error
    assert abs(float(C.sum()) - v0) <= 1e-2 * v0
    stt = st.cpu().numpy()
    iface = ((C > 0) & (C < 1)).cpu().numpy()
    assert np.all(np.isin(stt[iface], [1, 2, 3, 4, 5])) and np.all(stt[~iface] == 0)
    g.close()
    mlp.close()


def _windows(cb, count, W_, seed):
    """Window origins (z, y, x) centred on random marker nodes."""
    rng = np.random.default_rng(seed)
    c = (cb & 1)
    mark = (c != torch.roll(c, -1, dims=2)) | (c != torch.roll(c, -1, dims=1)) | (c != torch.roll(c, -1, dims=0))
    idx = torch.nonzero(mark.reshape(-1)).reshape(-1)
    pick = idx[torch.from_numpy(rng.choice(idx.numel(), size=count, replace=False)).cuda()].cpu().numpy()
    n = cb.shape[0]
    return [((p // (n * n)) - W_ // 2, ((p // n) % n) - W_ // 2, (p % n) - W_ // 2) for p in pick]


def _cut(t, o, W_):
    """Periodic window [o, o + W) of the last three axes of a device tensor."""
    n = t.shape[-1]
    iz, iy, ix = [(torch.arange(W_, device=t.device) + o[k]) % n for k in range(3)]
    return t.index_select(-3, iz).index_select(-2, iy).index_select(-1, ix).cpu().numpy()


def _present(cb):
    c = cb & 1
    return np.stack([c != np.roll(c, -1, axis=2), c != np.roll(c, -1, axis=1), c != np.roll(c, -1, axis=0)])


def test_512_windows_match_the_oracle():
    w = W.merging_drops(n=512, seed=5)
    g = ebit.Grid(*w.n3)
    g.init(dev(w.phi), dev(w.phi_faces), dev(w.s_exact))
    ud = [dev(w.u[d]) for d in range(3)]
    del w.phi, w.phi_faces, w.s_exact
    Wn, M = 32, 4
    lam = w.lam(0)
    for k, d in enumerate((0, 1, 2)):
        cb0, s0 = g.get_state()
        wins = _windows(cb0, 3, Wn, seed=10 + k)
        before = [(_cut(cb0, o, Wn), _cut(s0, o, Wn), _cut(ud[d], o, Wn)) for o in wins]
        del cb0, s0
        g.sweep(d, ud[d], lam * g.h)
        cb1, s1 = g.get_state()
        for o, (wcb, ws, wu) in zip(wins, before):
            ost, _ = oracle.sweep(oracle.State(wcb, ws), d, wu, lam)
            gcb, gs = _cut(cb1, o, Wn), _cut(s1, o, Wn)
            inner = (slice(M, Wn - M),) * 3
            assert np.array_equal(gcb[inner], ost.cb[inner]), f"sweep {d}: colours differ in window {o}"
            m = _present(gcb)[(slice(None),) + inner]
            diff = np.abs(gs[(slice(None),) + inner][m] - ost.s[(slice(None),) + inner][m])
            assert diff.size > 0 and diff.max() <= TOL, f"sweep {d}: offsets differ in window {o}"
        del cb1, s1
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    g.front2vof(C)
    g.curvature(C, kh, st)
    cb, s = g.get_state()
    for o in _windows(cb, 4, Wn, seed=20):
        oC, _ = oracle.front2vof(oracle.State(_cut(cb, o, Wn), _cut(s, o, Wn)))
        gC = _cut(C, o, Wn)
        inner = (slice(2, Wn - 2),) * 3
        assert np.max(np.abs(gC[inner] - oC[inner])) <= TOL
        okh, ost_ = oracle.hf_curvature(gC)
        inner = (slice(6, Wn - 6),) * 3
        assert np.array_equal(_cut(st, o, Wn)[inner], ost_[inner])
        assert np.max(np.abs(_cut(kh, o, Wn)[inner] - okh[inner])) <= TOL
    g.close()


def _box(cb, centre, half):
    """Phase-1 node colours in the box of half-width ``half`` around ``centre``
    (x, y, z in cells), periodic."""
    n = cb.shape[-1]
    o = [int(round(centre[2])) - half, int(round(centre[1])) - half, int(round(centre[0])) - half]
    return (_cut(cb, o, 2 * half) & 1).astype(bool), o


def test_512_windows_where_the_drops_touch():
    """The 512^3 merging drops: the step where the colour field joins them (two
    phase-1 components in a box around the gap become one) is found, the run is
    repeated up to the last state with two components, and the next two steps'
    sweeps, Front2VOF
    and height functions are checked against the oracle on windows centred on
    the point where the drops come closest."""
    w = W.merging_drops(n=512, seed=5)
    n = w.n3[0]
    e1, e2 = w.shapes
    gap_c = (e1.centre[0] + W._extent(e1, 0) + 4.0 / n) * n, 0.5 * n, 0.5 * n
    half = 64
    phi, faces, sx = dev(w.phi), dev(w.phi_faces), dev(w.s_exact)
    del w.phi, w.phi_faces, w.s_exact
    ud = [dev(w.u[d]) for d in range(3)]
    g = ebit.Grid(*w.n3)
    g.init(phi, faces, sx)
    merged = None
    for k in range(260):
        g.step(k, ud, w.lam(k) * g.h)
        if k >= 100 and k % 2 == 1:
            cb, _ = g.get_state()
            box, _ = _box(cb, gap_c, half)
            nc = ndimage.label(box)[1]
            if k == 101:
                assert nc == 2, nc
            if nc == 1:
                merged = k
                break
    assert merged is not None, "the drops did not merge"
    # the same run up to the last state seen with two components (after step
    # merged - 2); the drops join in step merged - 1 or merged
    g.init(phi, faces, sx)
    for k in range(merged - 1):
        g.step(k, ud, w.lam(k) * g.h)
    cb, _ = g.get_state()
    box, o = _box(cb, gap_c, half)
    lab, nc = ndimage.label(box)
    assert nc == 2
    da = ndimage.distance_transform_edt(lab != 1)
    db = ndimage.distance_transform_edt(lab != 2)
    p = np.unravel_index(np.argmin(da + db), box.shape)
    contact = [o[k] + p[k] for k in range(3)]  # z, y, x
    Wn, M = 32, 4
    wins = [(contact[0] + dz - Wn // 2, contact[1] + dy - Wn // 2, contact[2] + dx - Wn // 2)
            for dz, dy, dx in ((0, 0, 0), (6, 0, 0), (0, 6, 0), (0, 0, -6))]
    del cb
    for step in (merged - 1, merged):
        lam = w.lam(step)
        for d in ((0, 1, 2) if step % 2 == 0 else (2, 1, 0)):
            cb0, s0 = g.get_state()
            before = [(_cut(cb0, o_, Wn), _cut(s0, o_, Wn), _cut(ud[d], o_, Wn)) for o_ in wins]
            del cb0, s0
            g.sweep(d, ud[d], lam * g.h)
            cb1, s1 = g.get_state()
            for o_, (wcb, ws, wu) in zip(wins, before):
                ost, _ = oracle.sweep(oracle.State(wcb, ws), d, wu, lam)
                gcb, gs = _cut(cb1, o_, Wn), _cut(s1, o_, Wn)
                inner = (slice(M, Wn - M),) * 3
                assert np.array_equal(gcb[inner], ost.cb[inner]), f"step {step} sweep {d}: colours differ in {o_}"
                m = _present(gcb)[(slice(None),) + inner]
                diff = np.abs(gs[(slice(None),) + inner][m] - ost.s[(slice(None),) + inner][m])
                assert diff.size > 0 and diff.max() <= TOL, f"step {step} sweep {d}: offsets differ in {o_}"
            del cb1, s1
    cb, s = g.get_state()
    assert ndimage.label(_box(cb, gap_c, half)[0])[1] == 1  # the checked steps joined the drops
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    g.front2vof(C)
    g.curvature(C, kh, st)
    for o_ in wins:
        oC, _ = oracle.front2vof(oracle.State(_cut(cb, o_, Wn), _cut(s, o_, Wn)))
        gC = _cut(C, o_, Wn)
        inner = (slice(2, Wn - 2),) * 3
        assert np.max(np.abs(gC[inner] - oC[inner])) <= TOL
        okh, ost_ = oracle.hf_curvature(gC)
        inner = (slice(6, Wn - 6),) * 3
        assert np.array_equal(_cut(st, o_, Wn)[inner], ost_[inner])
        assert np.max(np.abs(_cut(kh, o_, Wn)[inner] - okh[inner])) <= TOL
    g.close()
