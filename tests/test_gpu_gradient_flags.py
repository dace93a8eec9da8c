"""The paper's flag rule (Eq. 2.8: gradient norm of the P1-interpolated
viscosity above nu on some finest element a coarse element covers) through
agca_flag_gradient, against the oracle: flags and flagged lists bit-exact
(both sides compare in FP64; the oracle takes the gradient from barycentric
gradients, the kernel from path differences, so the check first makes sure
no finest gradient lies within 1e-12 of nu), every level's apply to 1e-12."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from synth import random_vector, sphere_sinkers, sphere_sinkers_vertex

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


def test_gradient_flags_match_oracle():
    N, L, nu = 8, 3, 200.0
    p = sphere_sinkers(N, 3, 0.15, 0.02, 1e4)
    eta_v = sphere_sinkers_vertex(N, 3, 0.15, 0.02, 1e4)
    gmax, flags = oagca.gradient_flags(N, L, eta_v, nu)
    assert np.abs(gmax[L] - nu).min() > 1e-12 * nu
    assert 0 < flags[L - 1].sum() < flags[L - 1].size
    H = oagca.Hierarchy(N, L, p.eta, nu, eta_vertex=eta_v)
    c = pkg.Context(N, L, pkg.FP64, device=DEV)
    c.set_viscosity(torch.from_numpy(p.eta).to(DEV))
    c.flag_gradient(torch.from_numpy(eta_v).to(DEV), nu)
    c.setup()
    for l in range(1, L):
        got = c.level_data(l, pkg.FIELD_FLAGS).cpu().numpy().astype(bool)
        assert np.array_equal(got, flags[l]), l
        assert np.array_equal(c.level_data(l, pkg.FIELD_LIST).cpu().numpy(), np.nonzero(flags[l])[0]), l
        assert np.array_equal(c.level_data(l, pkg.FIELD_MEAN).cpu().numpy(), H.mean[l]), l
    for l in range(1, L + 1):
        x = random_vector(3 * c.V[l], 60 + l)
        got = c.apply(l, torch.from_numpy(x).to(DEV)).cpu().numpy()
        ref = H.A[l] @ (x * H.mask[l])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), l
