"""The allocation-free Stokes apply (agca_stokes_apply_static), for callers
that cannot allocate device memory, against the context-based
agca_stokes_apply on the same inputs, on two calls in a row.  This file is
collected last."""
import numpy as np
import pytest
import torch

from synth import random_vector, sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("N", [4, 8])
def test_static_apply_matches_context_apply(N):
    p = sphere_sinkers(N, 3, 0.15, 0.02, 1e6)
    eta = torch.from_numpy(p.eta).to(DEV)
    ctx = pkg.Context(N, device=DEV)
    ctx.set_viscosity(eta)
    for call in range(2):
        x = torch.from_numpy(random_vector(ctx.nt, 90 + call)).to(DEV)
        ref = ctx.stokes_apply(x)
        y = torch.full_like(x, float("nan"))  # the caller provides the output
        got = pkg.stokes_apply_static(N, eta, x, y)
        torch.cuda.synchronize()
        assert got.data_ptr() == y.data_ptr()
        err = float((got - ref).abs().max()) / float(ref.abs().max())
        assert err <= 1e-12, (call, err)


def test_static_apply_rejects_sizes_beyond_limit():
    N = pkg.agca.STATIC_MAX_N + 1
    nL = 2 * N
    eta = torch.ones(6 * nL ** 3, dtype=torch.float64, device=DEV)
    x = torch.zeros(3 * (nL + 1) ** 3 + (N + 1) ** 3, dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.AgcaError) as ei:
        pkg.stokes_apply_static(N, eta, x, torch.empty_like(x))
    assert ei.value.status == 1
