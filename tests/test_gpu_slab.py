"""The CUDA library as the per-rank engine of the z-slab decomposition
(paper_2509_26361_gb300/slab.py), through the C ABI: a one-rank slab, and two
slabs stepped in one process with their halos reloaded after every sweep, give
the owned layers of the single-domain oracle run bit for bit (colours) and to
1e-12 (offsets).  No kernel waits on another rank: the exchange is on the
host."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_26361_gb300 import slab as S

from test_slab import N3, _problem

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _present(cb):
    c = cb & 1
    return np.stack([c != np.roll(c, -1, 2), c != np.roll(c, -1, 1), c != np.roll(c, -1, 0)])


def _check(owned_cb, owned_s, ref_cb, ref_s):
    assert np.array_equal(owned_cb, ref_cb)
    m = (ref_s != 0.0) | (owned_s != 0.0)
    assert np.abs(owned_s[m] - ref_s[m]).max() <= TOL


def test_one_rank_slab_on_the_gpu():
    phi, faces, u, lams = _problem()
    st = oracle.init(phi, faces)
    sl = S.Slab(N3[2], 0, 1)
    eng = S.GridEngine((N3[0], N3[1], sl.nz_local), 1.0 / N3[0])
    cb = torch.from_numpy(sl.cut(st.cb)).cuda()
    s = torch.from_numpy(sl.cut(st.s)).cuda()
    ul = [torch.from_numpy(sl.cut(u[d])).cuda() for d in range(3)]
    cb, s = S.run_steps(sl, eng, cb, s, ul, lams)
    eng.close()
    for n, lam in enumerate(lams):
        st = oracle.step(st, n, u, lam)
    _check(sl.owned(cb.cpu().numpy()), sl.owned(s.cpu().numpy()), st.cb, st.s)


def test_two_slabs_on_the_gpu_with_reloaded_halos():
    phi, faces, u, lams = _problem()
    st0 = oracle.init(phi, faces)
    for rank in range(2):
        sl = S.Slab(N3[2], rank, 2)
        eng = S.GridEngine((N3[0], N3[1], sl.nz_local), 1.0 / N3[0])
        ul = [torch.from_numpy(sl.cut(u[d])).cuda() for d in range(3)]
        stg = st0
        cb = torch.from_numpy(sl.cut(stg.cb)).cuda()
        s = torch.from_numpy(sl.cut(stg.s)).cuda()
        for n, lam in enumerate(lams):
            for d in ((0, 1, 2) if n % 2 == 0 else (2, 1, 0)):
                cb, s = eng(cb, s, d, ul[d], lam)
                stg, _ = oracle.sweep(stg, d, u[d], lam)
                _check(sl.owned(cb.cpu().numpy()), sl.owned(s.cpu().numpy()), stg.cb[sl.z0:sl.z1],
                       stg.s[:, sl.z0:sl.z1])
                cb = torch.from_numpy(sl.cut(stg.cb)).cuda()
                s = torch.from_numpy(sl.cut(stg.s)).cuda()
        eng.close()
