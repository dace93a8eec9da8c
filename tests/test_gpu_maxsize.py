"""The largest grid the library accepts: 256^3 pressure cubes, 512^3 velocity
cubes, 8 levels, 405 M velocity DoF.  Element ids reach 8.05e8 and vector
offsets 4.05e8, the top of the kernels' 32-bit indexing.  Checked: finest
apply rows (FP64 and FP32) against the oracle's pointwise rows, including the
vertices with the largest ids; the mixed V-cycle symmetric and positive; a
mixed Stokes solve checked with an independent FP64 apply of the Stokes
operator.  Inputs stay on the device (the host copies of
the element fields would take 26 GB); the oracle reads the entries it needs
one by one.
"""
import numpy as np
import pytest
import torch

from oracle import pointwise
from synth import sphere_sinkers_on_device

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")
N = 256


class _Entries:
    """Host view of a device vector, read one entry at a time."""

    def __init__(self, t):
        self.t = t

    def __getitem__(self, i):
        return float(self.t[int(i)])


@pytest.fixture(scope="module")
def big():
    eta, fbar, centres = sphere_sinkers_on_device(N, 8, 0.08, 0.01, 1e3, device=DEV)
    ctx = pkg.Context(N, None, pkg.MIXED, device=DEV)
    assert ctx.L == 8
    ctx.prepare(eta, 10.0)
    b = ctx.load_vector(fbar.reshape(-1))
    del fbar
    return eta, centres, ctx, b


def test_fine_apply_rows_at_max_size(big):
    eta, centres, ctx, _ = big
    n, L = 2 * N, ctx.L
    m, V = n + 1, ctx.V[L]
    g = torch.Generator(device=DEV).manual_seed(31)
    x = torch.rand(3 * V, dtype=torch.float64, device=DEV, generator=g) * 2 - 1
    y64 = ctx.apply(L, x)
    x32 = x.float()
    y32 = ctx.apply(L, x32, dtype=pkg.F32)
    rng = np.random.default_rng(8)
    verts = list(rng.integers(0, V, 24))
    for ijk in ([n - 1, n - 1, n - 1], [n - 2, n - 1, n - 1], [1, 1, 1], [n - 1, 1, n - 1], [1, n - 1, n - 2],
                [n // 2, n // 2, n - 1], [0, 7, 7], [n, n, n]):
        verts.append(ijk[0] + m * (ijk[1] + m * ijk[2]))
    for c in centres[:3]:  # next to sinker surfaces
        ijk = np.clip(np.round((c + [0.08, 0, 0]) * n).astype(int), 1, n - 1)
        verts.append(ijk[0] + m * (ijk[1] + m * ijk[2]))
    verts = np.array(verts, dtype=np.int64)
    idx = torch.from_numpy(np.concatenate([c * V + verts for c in range(3)])).to(DEV)
    got64 = y64[idx].cpu().numpy().reshape(3, -1).T
    got32 = y32[idx].double().cpu().numpy().reshape(3, -1).T
    ref = pointwise.fine_rows(N, _Entries(eta), _Entries(x), verts)
    ref32 = pointwise.fine_rows(N, _Entries(eta), _Entries(x32), verts)
    assert np.abs(ref).max() > 0
    assert np.abs(got64 - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(got32 - ref32).max() <= 1e-5 * np.abs(ref32).max()
    vi, vj, vk = verts % m, (verts // m) % m, verts // (m * m)
    on_bnd = (np.minimum(np.minimum(vi, vj), vk) == 0) | (np.maximum(np.maximum(vi, vj), vk) == n)
    assert on_bnd.sum() >= 2 and not got64[on_bnd].any() and not got32[on_bnd].any()  # Dirichlet rows


def test_vcycle_symmetric_positive_at_max_size(big):
    _, _, ctx, _ = big
    n3 = 3 * ctx.V[ctx.L]
    g = torch.Generator(device=DEV).manual_seed(32)
    r1 = torch.rand(n3, dtype=torch.float64, device=DEV, generator=g) * 2 - 1
    r2 = r1 + 0.5 * (torch.rand(n3, dtype=torch.float64, device=DEV, generator=g) * 2 - 1)
    z1 = ctx.vcycle(r1)
    z2 = ctx.vcycle(r2)
    assert bool(torch.isfinite(z1).all()) and bool(torch.isfinite(z2).all())
    a, b = float(torch.dot(z1, r2)), float(torch.dot(r1, z2))
    assert float(torch.dot(z1, r1)) > 0 and a > 0
    # FP32 cycle: symmetric up to single-precision rounding
    assert abs(a - b) <= 1e-4 * abs(a)


def test_mixed_solve_at_max_size(big):
    _, _, ctx, b = big
    x, its, rel = ctx.solve(b, 1e-3, 3000)
    assert rel <= 1e-3 and its > 0
    r = b - ctx.stokes_apply(x)
    true_rel = float(torch.linalg.vector_norm(r)) / float(torch.linalg.vector_norm(b))
    assert true_rel <= 1.01e-3
    pr = x[3 * ctx.V[ctx.L]:]
    assert abs(float(pr.mean())) <= 1e-12 * float(pr.abs().max())
