"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Bar (from the method's data): colour bytes, topology counters and statuses
bit-exact; FP64 marker offsets, volume fractions and curvature within 1e-12
absolute.  Offsets are compared on edges that carry a marker (the offset of an
empty edge is unspecified and reads back as 0).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def present_mask(cb):
    c = cb & 1
    return np.stack([c != np.roll(c, -1, axis=2), c != np.roll(c, -1, axis=1), c != np.roll(c, -1, axis=0)])


def compare_state(g, ost, where=""):
    cb, s = g.get_state()
    cb = cb.cpu().numpy()
    s = s.cpu().numpy()
    assert np.array_equal(cb, ost.cb), f"colour bytes differ {where}: {np.argwhere(cb != ost.cb)[:5]}"
    m = present_mask(cb)
    d = np.abs(s[m] - ost.s[m])
    assert d.size == 0 or d.max() <= TOL, f"offsets differ {where}: {d.max()}"
    assert np.all(s[~m] == 0.0)
    return cb, s


def run_pair(n3, phi, faces, u, lams, steps, s_exact=None, dense=False, check_every=1, f2v=True, hf=True):
    nx, ny, nz = n3
    g = ebit.Grid(nx, ny, nz, h=1.0 / nx, dense=dense)
    g.init(to_dev(phi), None if faces is None else to_dev(faces), None if s_exact is None else to_dev(s_exact))
    ost = oracle.init(phi, faces, s_exact)
    compare_state(g, ost, "after init")
    ud = [to_dev(u[d]) for d in range(3)]
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    ocnt = np.zeros(5, np.int64)
    for n in range(steps):
        order = (0, 1, 2) if n % 2 == 0 else (2, 1, 0)
        for d in order:
            lam = lams(n)
            dt = lam * g.h
            g.sweep(d, ud[d], dt)
            ost, c = oracle.sweep(ost, d, u[d], dt / g.h)
            ocnt += c
            if (n % check_every) == 0:
                compare_state(g, ost, f"step {n} dir {d}")
        if f2v:
            g.front2vof(C)
            oC, nbad = oracle.front2vof(ost)
            assert nbad == 0
            dC = np.abs(C.cpu().numpy() - oC).max()
            assert dC <= TOL, f"C differs at step {n}: {dC}"
            if hf:
                g.curvature(C, kh, st)
                okh, ost_ = oracle.hf_curvature(oC)
                assert np.array_equal(st.cpu().numpy(), ost_), f"HF status differs at step {n}"
                dk = np.abs(kh.cpu().numpy() - okh).max()
                assert dk <= TOL, f"kappa differs at step {n}: {dk}"
    compare_state(g, ost, "final")
    cnt = g.counters()
    assert [cnt[k] for k in ebit.COUNTER_NAMES] == list(ocnt), (cnt, ocnt)
    assert cnt["tiles"] > 0
    g.close()
    return ost


def blobs(n3, seed, count, rmin, rmax):
    rng = np.random.default_rng(seed)
    sp = [W.Sphere(tuple(rng.uniform(0, 1, 3)), rng.uniform(rmin, rmax)) for _ in range(count)]
    return W.sphere_phi_nodes_faces(n3, sp)


@pytest.mark.parametrize("dense", [False, True])
def test_translation_sphere_exact_roots(dense):
    w = W.translation_sphere(32)
    run_pair(w.n3, w.phi, w.phi_faces, w.u, lambda n: 0.25, 8, s_exact=w.s_exact, dense=dense)


@pytest.mark.parametrize("seed", [1, 2])
def test_fourier_spheres_small(seed):
    w = W.fourier_spheres(n=32, seed=seed, count=4, rmin=0.06, rmax=0.14, steps=6)
    run_pair(w.n3, w.phi, w.phi_faces, w.u, w.lam, w.steps)


@pytest.mark.parametrize("seed", [61, 62])
def test_gyroid_surfaces_with_saddle_faces(seed):
    """Smooth triply periodic surfaces whose faces include saddles (diagonal
    corners on the same side), exact edge roots, a Fourier field: the saddle
    face colours and segment pairings of every sweep against the oracle."""
    rng = np.random.default_rng(seed)
    n = 16
    phi, faces, roots = W.gyroid_surface(n, rng.integers(4, 6, size=3), rng.uniform(0.0, 2.0 * np.pi, size=3),
                                         rng.uniform(-0.3, 0.3))
    u = W.fourier_velocity((n, n, n), rng)
    run_pair((n, n, n), phi, faces, u, lambda k: 0.5, 4, s_exact=roots)


@pytest.mark.parametrize("n3", [(20, 24, 28), (9, 17, 8)])
def test_ragged_grid_random_blobs(n3):
    """Grids that are not multiples of the 8-cell tile, lumpy shapes with thin
    features (topology changes, saddle faces) in a seeded divergence-free field."""
    rng = np.random.default_rng(7)
    phi, faces = blobs(n3, 3, 9, 0.04, 0.12)
    u = W.fourier_velocity(n3, rng)
    run_pair(n3, phi, faces, u, lambda n: 0.9 if n % 3 else -0.7, 6)


def test_empty_and_full_domains():
    for val in (-1.0, 1.0):
        n3 = (16, 16, 16)
        phi = np.full((16, 16, 16), val)
        u = W.fourier_velocity(n3, np.random.default_rng(1))
        run_pair(n3, phi, None, u, lambda n: 0.5, 2)


def test_band_matches_dense_over_many_steps():
    w = W.fourier_spheres(n=48, seed=5, count=5, rmin=0.05, rmax=0.11)
    res = []
    for dense in (False, True):
        g = ebit.Grid(48, 48, 48, dense=dense)
        g.init(to_dev(w.phi), to_dev(w.phi_faces))
        ud = [to_dev(w.u[d]) for d in range(3)]
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        kh = torch.zeros_like(C)
        st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
        for n in range(40):
            g.step(n, ud, w.lam(n) * g.h)
            g.front2vof(C)
            g.curvature(C, kh, st)
        cb, s = g.get_state()
        res.append((cb.cpu().numpy(), s.cpu().numpy(), C.cpu().numpy(), kh.cpu().numpy(), st.cpu().numpy()))
        g.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_full_size_config_sampled_steps():
    """128^3, 8 spheres, 12-mode field: the benchmark's launch configuration (band
    mode); a few steps compared whole-array with the oracle."""
    w = W.fourier_spheres(n=128, seed=2)
    run_pair(w.n3, w.phi, w.phi_faces, w.u, w.lam, 2, check_every=1)


def test_errors_are_reported():
    g = ebit.Grid(16, 16, 16)
    u = torch.ones(g.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ebit.EbitError) as e:
        g.sweep(3, u, 0.01)
    assert e.value.code == ebit.EBIT_EINVAL
    with pytest.raises(ebit.EbitError) as e:
        g.sweep(0, u, float("nan"))
    assert e.value.code == ebit.EBIT_ENONFINITE
    phi, faces = blobs((16, 16, 16), 1, 3, 0.15, 0.3)
    g.init(to_dev(phi), to_dev(faces))
    g.sweep(0, u, 1.5 * g.h)  # markers move 1.5 cells: clamped on the device, raised at sync
    with pytest.raises(ebit.EbitError) as e:
        g.sync()
    assert e.value.code == ebit.EBIT_ECFL
    g.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_velocity_is_reported_before_cfl(bad):
    """A NaN or infinite velocity where a marker samples it is named as such
    (EBIT_ENONFINITE), not as a CFL violation, even when the same sweep also
    moves markers a full cell; the markers it touches stay in place.  A
    non-finite value that no marker samples is harmless."""
    n3 = (16, 16, 16)
    phi, faces = blobs(n3, 1, 3, 0.15, 0.3)
    g = ebit.Grid(*n3)
    g.init(to_dev(phi), to_dev(faces))
    cb0, _ = g.get_state()
    c = cb0.cpu().numpy() & 1
    xm = np.argwhere(c != np.roll(c, -1, axis=2))  # nodes owning an x-edge marker
    offs = [(dz, dy, dx) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)]
    far = np.argwhere(np.all([np.roll(c, o, axis=(0, 1, 2)) == c for o in offs], axis=0))
    u = torch.full(g.shape, 0.3, dtype=torch.float64, device="cuda")
    # a face whose 5x5x5 node neighbourhood holds no colour change: no marker
    # interpolates there (the trilinear stencil reaches one face further)
    k, j, i = far[0]
    u[k, j, i] = bad
    g.sweep(0, u, g.h)
    assert g.sync() == ebit.EBIT_OK
    assert g.counters()["nonfinite"] == 0
    # every marker moves 1.5 cells, and the faces one marker samples are bad
    u = torch.full(g.shape, 1.5, dtype=torch.float64, device="cuda")
    k, j, i = xm[0]
    u[k, j, i] = bad
    u[k, j, (i + 1) % n3[0]] = bad
    g.sweep(0, u, g.h)
    with pytest.raises(ebit.EbitError) as e:
        g.sync()
    assert e.value.code == ebit.EBIT_ENONFINITE
    with pytest.raises(ebit.EbitError) as e:
        g.counters()
    assert e.value.code == ebit.EBIT_ENONFINITE
    # after a reset the context works again
    g.reset_counters()
    g.init(to_dev(phi), to_dev(faces))
    g.sweep(0, torch.full(g.shape, 0.3, dtype=torch.float64, device="cuda"), g.h)
    assert g.sync() == ebit.EBIT_OK
    g.close()


def random_state(n3, seed):
    """Any colour field is a valid EBIT state: markers where node colours differ,
    face colours used on saddle faces.  Random fields reach every local corner
    and face configuration, including saddles and several loops per cell."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n3
    cb = rng.integers(0, 16, size=(nz, ny, nx), dtype=np.uint8)
    s = rng.uniform(0.0, 1.0, size=(3, nz, ny, nx))
    st = oracle.State(cb, s)
    # canonical form: offsets 0 where no marker, face colour = lowest corner except saddles
    c = cb & 1
    pres = present_mask(cb)
    s[~pres] = 0.0
    for a in range(3):
        ax1, ax2 = [b for b in range(3) if b != a]
        sh = lambda arr, b: np.roll(arr, -1, axis=2 - b)
        c10, c01 = sh(c, ax1), sh(c, ax2)
        c11 = sh(c10, ax2)
        sad = (c == c11) & (c10 == c01) & (c != c10)
        bit = np.where(sad, (cb >> (1 + a)) & 1, c)
        cb = (cb & ~np.uint8(1 << (1 + a))) | (bit.astype(np.uint8) << (1 + a))
    st.cb = np.ascontiguousarray(cb)
    st.s = np.ascontiguousarray(s)
    return st


@pytest.mark.parametrize("seed", [11, 12])
def test_front2vof_hf_random_colour_fields(seed):
    n3 = (16, 16, 16)
    st = random_state(n3, seed)
    g = ebit.Grid(*n3)
    g.set_state(to_dev(st.cb), to_dev(st.s))
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    stt = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    g.front2vof(C, ebit.EBIT_FULL)
    oC, nbad = oracle.front2vof(st)
    assert nbad == 0
    assert np.abs(C.cpu().numpy() - oC).max() <= TOL
    g.curvature(C, kh, stt, flags=ebit.EBIT_FULL)
    okh, ost = oracle.hf_curvature(oC)
    assert np.array_equal(stt.cpu().numpy(), ost)
    assert np.abs(kh.cpu().numpy() - okh).max() <= TOL
    g.close()


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_sweeps_on_random_colour_fields(seed):
    """Sweeps from random states: saddles everywhere, many annihilations and
    multi-crossings; every rule against the oracle."""
    n3 = (12, 16, 20)
    st = random_state(n3, seed)
    rng = np.random.default_rng(seed)
    u = W.fourier_velocity(n3, rng)
    g = ebit.Grid(*n3)
    g.set_state(to_dev(st.cb), to_dev(st.s))
    ud = [to_dev(u[d]) for d in range(3)]
    ocnt = np.zeros(5, np.int64)
    ost = st
    for k, d in enumerate((0, 1, 2, 2, 1, 0)):
        dt = (0.93 if k % 2 == 0 else -0.61) * g.h
        g.sweep(d, ud[d], dt)
        ost, c = oracle.sweep(ost, d, u[d], dt / g.h)
        ocnt += c
        compare_state(g, ost, f"sweep {k} dir {d}")
    cnt = g.counters()
    assert [cnt[k] for k in ebit.COUNTER_NAMES] == list(ocnt), (cnt, ocnt)
    g.close()


def _hf_case(C):
    """Height functions of an arbitrary fraction field (full scan) against the oracle."""
    nz, ny, nx = C.shape
    g = ebit.Grid(nx, ny, nz)
    Cd = to_dev(C)
    kh = torch.zeros_like(Cd)
    stt = torch.zeros(Cd.shape, dtype=torch.uint8, device="cuda")
    g.curvature(Cd, kh, stt, flags=ebit.EBIT_FULL)
    okh, ost = oracle.hf_curvature(C)
    assert np.array_equal(stt.cpu().numpy(), ost)
    assert np.abs(kh.cpu().numpy() - okh).max() <= TOL
    g.close()
    return ost


def test_hf_normal_ties_and_ranges():
    """Fields where the float normal cannot decide: a grid-aligned slab (two
    normal components exactly zero), a diagonal plane (|n_x| = |n_y| exactly,
    ties to the lower axis), and fractions outside [0, 1]; the FP64 sums must
    give the oracle's statuses and curvature."""
    n = 16
    z = np.arange(n)[:, None, None] * np.ones((1, n, n))
    slab = np.where((z >= 2) & (z < 7), 1.0, 0.0)
    slab[7] = 0.3
    slab[1] = 0.6
    st = _hf_case(slab)
    assert np.all(st[7] == 3) and np.all(st[1] == 3)  # columns along z
    x = np.arange(n)[None, None, :] * np.ones((n, n, 1))
    y = np.arange(n)[None, :, None] * np.ones((n, 1, n))
    d = (x + y + 0.5) / np.sqrt(2.0) - 10.0 / np.sqrt(2.0)  # plane x + y = 9.5
    diag = np.clip(0.5 - d, 0.0, 1.0)
    st = _hf_case(diag)
    assert np.any(st == 1)  # ties resolved to the lower axis, as the oracle does
    rng = np.random.default_rng(5)
    wild = np.clip(slab + rng.normal(0.0, 0.05, slab.shape), -0.2, 1.2)
    wild[(wild > 0.0) & (wild < 1.0) & (z != 7) & (z != 1)] = 1.0
    _hf_case(wild)


def test_checkpoint_resume_is_bit_identical():
    """Run 2k steps in one context; run k steps in another, read its state back
    to the host, restore it into a fresh context and run k more: colour bytes
    and offsets are identical bit for bit (the restored context's first sweep
    processes every tile, the continuous one only its band)."""
    w = W.fourier_spheres(n=40, seed=5, count=5, rmin=0.07, rmax=0.15, steps=12)
    k = 6
    ud = [to_dev(w.u[d]) for d in range(3)]
    a = ebit.Grid(*w.n3)
    a.init(to_dev(w.phi), to_dev(w.phi_faces))
    for n in range(2 * k):
        a.step(n, ud, w.lam(n) * a.h)
    cb_a, s_a = (t.cpu().numpy() for t in a.get_state())
    b = ebit.Grid(*w.n3)
    b.init(to_dev(w.phi), to_dev(w.phi_faces))
    for n in range(k):
        b.step(n, ud, w.lam(n) * b.h)
    cb_h, s_h = (t.cpu().numpy() for t in b.get_state())
    b.close()
    c = ebit.Grid(*w.n3)
    c.set_state(torch.from_numpy(cb_h).cuda(), torch.from_numpy(s_h).cuda())
    for n in range(k, 2 * k):
        c.step(n, ud, w.lam(n) * c.h)
    cb_c, s_c = (t.cpu().numpy() for t in c.get_state())
    assert np.array_equal(cb_a, cb_c)
    assert np.array_equal(s_a.view(np.uint64), s_c.view(np.uint64))
    assert present_mask(cb_a).sum() > 1000
    a.close()
    c.close()


def test_async_front2vof_and_curvature_match_the_ordered_calls():
    """Front2VOF and curvature on the side stream (EBIT_ASYNC), overlapping the
    next step's sweeps, give the same fractions, curvature and statuses at
    every step as ordered calls, read the way a host copy would read them
    (another stream waits on ebit_event_record while the sweeps go on); the
    state after the last step is identical; async and ordered calls mix."""
    w = W.fourier_spheres(n=40, seed=6, count=5, rmin=0.07, rmax=0.15, steps=8)
    ud = [to_dev(w.u[d]) for d in range(3)]
    steps = 8
    res = []
    for asynch in (False, True):
        g = ebit.Grid(*w.n3)
        g.init(to_dev(w.phi), to_dev(w.phi_faces))
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        kh = torch.zeros_like(C)
        st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
        g.front2vof(C, ebit.EBIT_FULL)
        g.curvature(C, kh, st, flags=ebit.EBIT_FULL)
        snaps = []
        copy = torch.cuda.Stream()
        done = None
        for n in range(steps):
            g.step(n, ud, w.lam(n) * g.h)
            # the previous step's copies finish before Front2VOF overwrites C
            # (the sweeps above did not wait for them)
            if done is not None:
                torch.cuda.current_stream().wait_event(done)
            # step 5 mixes in ordered calls
            fl = ebit.EBIT_ASYNC if (asynch and n != 5) else ebit.EBIT_INCREMENTAL
            g.front2vof(C, fl)
            g.curvature(C, kh, st, flags=fl)
            ev = torch.cuda.Event()
            g.record_done(ev)
            with torch.cuda.stream(copy):
                copy.wait_event(ev)
                snaps.append((C.clone(), kh.clone(), st.clone()))
                done = torch.cuda.Event()
                done.record(copy)
        g.join()
        torch.cuda.synchronize()
        cb, s = g.get_state()
        res.append(([tuple(t.cpu().numpy() for t in sn) for sn in snaps], cb.cpu().numpy(), s.cpu().numpy(),
                    g.counters()))
        g.close()
    (sa, cba, sa_s, ca), (sb, cbb, sb_s, cbc) = res
    for n in range(steps):
        for x, y in zip(sa[n], sb[n]):
            assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), f"step {n}"
    assert np.array_equal(cba, cbb) and np.array_equal(sa_s.view(np.uint64), sb_s.view(np.uint64))
    assert ca == cbc
