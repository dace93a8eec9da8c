"""Parity on the largest single-GPU workload: 128^3 pressure cubes (256^3
velocity cubes, 50.9 M velocity DoF), 20 Gaussian log-viscosity bumps
clipped to [1e-3, 1e3], 7 levels, mixed precision.  Flags and the viscosity
hierarchy bit-exact against the oracle at every level, the finest-level
apply on sampled rows computed one by one by the oracle, and a mixed solve
that reaches the 1e-8 residual on the true FP64 operator.
"""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from oracle import pointwise
from synth import gaussian_logbumps, random_vector

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")
N = 128


@pytest.fixture(scope="module")
def big():
    p = gaussian_logbumps(N, device=DEV)
    L = pkg.default_levels(N)
    eta = torch.from_numpy(p.eta).to(DEV)
    ctx = pkg.Context(N, L, pkg.MIXED, device=DEV)
    ctx.prepare(eta, 10.0)
    return p, L, eta, ctx


def test_flags_bit_exact(big):
    p, L, eta, ctx = big
    mean, mx, mn, flags = oagca.flag_hierarchy(N, L, p.eta, 10.0)
    for l in range(1, L):
        assert np.array_equal(ctx.level_data(l, pkg.FIELD_MEAN).cpu().numpy(), mean[l])
        assert np.array_equal(ctx.level_data(l, pkg.FIELD_FLAGS).cpu().numpy().astype(bool), flags[l])
        assert np.array_equal(ctx.level_data(l, pkg.FIELD_LIST).cpu().numpy(), np.nonzero(flags[l])[0])
    assert sum(ctx.level_info(l).n_flag for l in range(1, L)) > 0


def test_fine_apply_sampled_rows(big):
    p, L, eta, ctx = big
    n = 2 * N
    V = ctx.V[L]
    x = random_vector(3 * V, 91)
    y64 = ctx.apply(L, torch.from_numpy(x).to(DEV)).cpu().numpy()
    rng = np.random.default_rng(9)
    m = n + 1
    verts = list(rng.integers(0, m ** 3, 40))
    for c in p.meta["centres"][:6]:  # bump centres: largest viscosity gradients
        ijk = np.clip(np.round(np.asarray(c) * n).astype(int), 1, n - 1)
        verts.append(ijk[0] + m * (ijk[1] + m * ijk[2]))
    verts += [1 + m * (1 + m), (n - 1) + m * (n // 2 + m * 1), 0]
    verts = np.array(verts)
    ref = pointwise.fine_rows(N, p.eta, x, verts)
    got = np.stack([y64[c * V + verts] for c in range(3)], axis=1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_mixed_solve_reaches_tolerance(big):
    p, L, eta, ctx = big
    b = ctx.load_vector(torch.from_numpy(p.fbar.ravel()).to(DEV))
    x, its, rel = ctx.solve(b, 1e-8, 20000)
    assert rel <= 1e-8
    r = b - ctx.stokes_apply(x)  # FP64 Stokes operator, pinned in test_gpu_parity
    assert float(torch.linalg.vector_norm(r)) <= 1e-8 * float(torch.linalg.vector_norm(b)) * 1.01
