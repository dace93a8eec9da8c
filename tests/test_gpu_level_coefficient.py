"""Coarse DCA coefficients evaluated on the coarse grid itself (Eq. 2.5 with
the coefficient approximations of Sec. 3.2: the analytic viscosity at the
coarse element's quadrature points, or the mean of its P1 interpolant),
passed through agca_set_level_coefficient, against the oracle built with the
same level coefficients: every level's apply to 1e-12 (FP64) / 1e-5 (FP32
cycle), flags unchanged, and a solve to the true-residual tolerance."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from synth import cube_field, field_problem, level_coefficients, p1_element_means, random_vector

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("mode", ["analytic", "p1"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_level_coefficients_match_oracle(mode, prec):
    N, L = 8, 3
    fn = cube_field("tanh", 1e4, omega=20.0)
    p = field_problem(N, fn)
    eta = p.eta if mode == "analytic" else p1_element_means(2 * N, fn)
    lc = level_coefficients(fn, N, L, mode)
    H = oagca.Hierarchy(N, L, eta, 10.0, level_coef=lc)
    assert sum(len(H.flist[l]) for l in range(1, L)) > 0
    c = pkg.Context(N, L, pkg.FP64 if prec == "fp64" else pkg.MIXED, device=DEV)
    c.set_viscosity(torch.from_numpy(eta).to(DEV))
    c.flag(10.0)
    for l in range(1, L):
        c.set_level_coefficient(l, torch.from_numpy(lc[l]).to(DEV))
    c.setup()
    for l in range(1, L):
        assert np.array_equal(c.level_data(l, pkg.FIELD_MEAN).cpu().numpy(), lc[l])
        assert np.array_equal(c.level_data(l, pkg.FIELD_FLAGS).cpu().numpy().astype(bool), H.flags[l])
    for l in range(1, L + 1):
        x = random_vector(3 * c.V[l], 60 + l)
        if prec == "fp64":
            got = c.apply(l, torch.from_numpy(x).to(DEV)).cpu().numpy()
            ref = H.A[l] @ (x * H.mask[l])
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), l
        else:
            x32 = x.astype(np.float32)
            got = c.apply(l, torch.from_numpy(x32).to(DEV), dtype=pkg.F32).cpu().numpy().astype(np.float64)
            ref = H.A[l] @ (x32.astype(np.float64) * H.mask[l])
            assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), l
    b = c.load_vector(torch.from_numpy(p.fbar.ravel()).to(DEV))
    x, its, rel = c.solve(b, 1e-8, 20000)
    assert rel <= 1e-8


def test_level_coefficient_call_order_and_values():
    N, L = 4, 2
    c = pkg.Context(N, L, pkg.FP64, device=DEV)
    eta = torch.ones(c.E[L], dtype=torch.float64, device=DEV)
    coef = torch.ones(c.E[1], dtype=torch.float64, device=DEV)
    import ctypes

    lib = pkg.lib()
    c.set_viscosity(eta)
    # before agca_flag: AGCA_ESTATE (7); the finest level is not a coarse level: AGCA_EINVAL (1)
    assert lib.agca_set_level_coefficient(c._h, 1, ctypes.c_void_p(coef.data_ptr())) == 7
    c.flag(10.0)
    assert lib.agca_set_level_coefficient(c._h, L, ctypes.c_void_p(coef.data_ptr())) == 1
    bad = coef.clone()
    bad[3] = -1.0
    assert lib.agca_set_level_coefficient(c._h, 1, ctypes.c_void_p(bad.data_ptr())) == 1
    assert lib.agca_set_level_coefficient(c._h, 1, ctypes.c_void_p(coef.data_ptr())) == 0
