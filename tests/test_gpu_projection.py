"""Coarse DCA coefficient as the harmonic or geometric mean of the children
(the P0 projections of Sec. 3.2) against the oracle: the viscosity hierarchy
(harmonic bit-exact, since reciprocals, the pairwise sums and the final
division are correctly rounded on both sides; geometric to 1e-14, since log
and exp may differ by an ulp between the two math libraries), the flags
(bit-exact, they do not depend on the projection) and every level's apply
to 1e-12."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from synth import random_vector, sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("name", ["harmonic", "geometric"])
def test_coarse_projection_matches_oracle(name):
    kind = {"harmonic": pkg.PROJ_HARMONIC, "geometric": pkg.PROJ_GEOMETRIC}[name]
    N, L = 8, 3
    p = sphere_sinkers(N, 3, 0.15, 0.02, 1e4)
    H = oagca.Hierarchy(N, L, p.eta, 10.0, projection=name)
    c = pkg.Context(N, L, pkg.FP64, device=DEV)
    c.set_viscosity(torch.from_numpy(p.eta).to(DEV))
    c.set_coarse_projection(kind)
    c.flag(10.0)
    c.setup()
    for l in range(1, L):
        got = c.level_data(l, pkg.FIELD_MEAN).cpu().numpy()
        if name == "harmonic":
            assert np.array_equal(got, H.mean[l]), l
        else:
            assert np.allclose(got, H.mean[l], rtol=1e-14, atol=0), l
        assert np.array_equal(c.level_data(l, pkg.FIELD_FLAGS).cpu().numpy().astype(bool), H.flags[l])
    assert sum(len(H.flist[l]) for l in range(1, L)) > 0
    for l in range(1, L + 1):
        x = random_vector(3 * c.V[l], 40 + l)
        got = c.apply(l, torch.from_numpy(x).to(DEV)).cpu().numpy()
        ref = H.A[l] @ (x * H.mask[l])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), l
