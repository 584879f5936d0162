"""One-fluid coupling terms (Sec. 2.5, Eq. 6 and the continuum surface force)
on the CUDA path against the oracle, through the C ABI: the properties and the
face-centred force are the oracle's values on fractions and curvatures that
the library itself produced (height functions, and the network with its
height-function fallback), on a cubic and a ragged grid."""
import numpy as np
import pytest
import torch

from oracle import coupling as CP
from paper_2509_26361_gb300 import ebit, learned
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n3,mode", [((48, 48, 48), ebit.EBIT_CURV_HF), ((20, 24, 28), ebit.EBIT_CURV_HF),
                                     ((48, 48, 48), ebit.EBIT_CURV_MLP_HF)])
def test_terms_match_the_oracle(n3, mode):
    rng = np.random.default_rng(8)
    rmin = 3.0 / min(n3)
    sp = W.random_spheres(rng, 2, rmin, max(0.2, rmin + 0.05), min(n3))
    phi, faces = W.sphere_phi_nodes_faces(n3, sp)
    u = [dev(v) for v in W.fourier_velocity(n3, rng)]
    g = ebit.Grid(*n3)
    mlp = None
    if mode != ebit.EBIT_CURV_HF:
        mlp = learned.load_network()
        g.set_mlp(mlp)
    g.init(dev(phi), dev(faces))
    for k in range(3):
        g.step(k, u, 0.5 * g.h)
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    kh = torch.zeros_like(C)
    st = torch.zeros(g.shape, dtype=torch.uint8, device="cuda")
    g.front2vof(C, ebit.EBIT_FULL)
    g.curvature(C, kh, st, mode=mode, flags=ebit.EBIT_FULL)
    args = dict(sigma=0.072, rho1=998.0, rho2=1.2, mu1=1.0e-3, mu2=1.8e-5)
    rho, mu, f = g.one_fluid(C, kh, st, **args)
    Ch, khh, sth = C.cpu().numpy(), kh.cpu().numpy(), st.cpu().numpy()
    rho_r, mu_r = CP.properties(Ch, args["rho1"], args["rho2"], args["mu1"], args["mu2"])
    f_r = CP.csf_force(Ch, khh, sth, g.h, args["sigma"])
    assert np.array_equal(rho.cpu().numpy(), rho_r) and np.array_equal(mu.cpu().numpy(), mu_r)
    assert np.array_equal(f.cpu().numpy(), f_r)
    assert np.abs(f_r).max() > 0
    if mode == ebit.EBIT_CURV_MLP_HF:
        assert (sth == 5).any()  # the network's cells enter the face curvatures
    g.close()
    if mlp is not None:
        mlp.close()
