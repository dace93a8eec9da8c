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


# N = 32 is the limit: the divergence field then fills the second half of the
# scratch array to its last entry
@pytest.mark.parametrize("N", [4, 8, 32])
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


def test_static_apply_on_a_side_stream():
    """Two calls in a row on a caller's own stream, synchronising only that
    stream before reading the results."""
    N = 8
    p = sphere_sinkers(N, 3, 0.15, 0.02, 1e6)
    eta = torch.from_numpy(p.eta).to(DEV)
    ctx = pkg.Context(N, device=DEV)
    ctx.set_viscosity(eta)
    side = torch.cuda.Stream(device=DEV)
    xs = [torch.from_numpy(random_vector(ctx.nt, 120 + c)).to(DEV) for c in range(2)]
    refs = [ctx.stokes_apply(x) for x in xs]
    torch.cuda.synchronize()
    ys = [torch.full_like(x, float("nan")) for x in xs]
    for x, y in zip(xs, ys):
        pkg.stokes_apply_static(N, eta, x, y, stream=side)
    side.synchronize()
    for c, (y, ref) in enumerate(zip(ys, refs)):
        err = float((y - ref).abs().max()) / float(ref.abs().max())
        assert err <= 1e-12, (c, err)


def test_static_apply_rejects_host_memory():
    N = 4
    nL = 2 * N
    nt = 3 * (nL + 1) ** 3 + (N + 1) ** 3
    eta = torch.ones(6 * nL ** 3, dtype=torch.float64, device=DEV)
    x = torch.zeros(nt, dtype=torch.float64, device=DEV)
    y = torch.zeros(nt, dtype=torch.float64, device=DEV)
    host = torch.zeros(nt, dtype=torch.float64)
    import ctypes
    st = pkg.lib().agca_stokes_apply_static(N, ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(host.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(0))
    assert st == 1  # AGCA_EINVAL: x is not device memory of the current device
    del x


def test_static_apply_rejects_sizes_beyond_limit():
    N = pkg.agca.STATIC_MAX_N + 1
    nL = 2 * N
    eta = torch.ones(6 * nL ** 3, dtype=torch.float64, device=DEV)
    x = torch.zeros(3 * (nL + 1) ** 3 + (N + 1) ** 3, dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.AgcaError) as ei:
        pkg.stokes_apply_static(N, eta, x, torch.empty_like(x))
    assert ei.value.status == 1
