"""The paper's outer solver on the GPU (Sec. 4): FGMRES with the
block-triangular preconditioner of Eq. 4.1, Schur block the lumped 1/eta mass
or the diag(A)-BFBT of Eq. 4.2, against the oracle's FGMRES with the same
blocks (oracle.fgmres): the same iteration count (the GPU V-cycle equals the
oracle's to rounding; with enough conjugate-gradient steps the GPU's Z^-1
equals the oracle's sparse direct one) and the solution of the sparse direct
solve; at 8^3 pressure cubes the FGMRES and MINRES solutions agree."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from oracle import fgmres as ofg
from oracle import stokes as ostokes
from synth import sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def small():
    p = sphere_sinkers(4, 3, 0.15, 0.03, 1e4)
    H = oagca.Hierarchy(4, 2, p.eta, 10.0)
    S = ostokes.Stokes(H)
    c = pkg.Context(4, 2, pkg.FP64, device=DEV)
    c.prepare(torch.from_numpy(p.eta).to(DEV), 10.0)
    b = c.load_vector(torch.from_numpy(p.fbar.ravel()).to(DEV))
    bo = S.rhs(p.fbar)
    assert np.abs(b.cpu().numpy() - bo).max() <= 1e-14 * np.abs(bo).max()   # summation order
    return p, S, c, b, bo


@pytest.mark.parametrize("schur", ["mass", "bfbt"])
def test_fgmres_matches_oracle(small, schur):
    p, S, c, b, bo = small
    if schur == "mass":
        Q = ofg.BlockTriangular(S, s_inv=lambda rp: S.project(S.project(rp) / S.Mp))
    else:
        Q = ofg.BlockTriangular(S)
    xo, itso = ofg.solve(S, bo, rtol=1e-10, restart=50, maxit=2000, precond=Q)
    x, its, rel = c.solve_fgmres(b, 1e-10, 2000, restart=50, schur=schur, z_iters=300)
    assert rel <= 1e-10
    assert abs(its - itso) <= 1, (its, itso)
    xg = x.cpu().numpy()
    # the oracle's own operator confirms the residual; the error against the
    # direct solve is bounded by cond(K) times the residual (jump 1e4 here:
    # about 4e-8 measured with the mass Schur block)
    assert np.linalg.norm(bo - S.K(xg)) <= 1.01e-10 * np.linalg.norm(bo)
    xd = S.direct(bo)
    err = np.abs(xg - xd).max() / np.abs(xd).max()
    print(f"\n4^3 FGMRES ({schur}) {its} iterations: error against the direct solve {err:.1e}")
    assert err <= 1e-6


def test_fgmres_restarts_and_agrees_with_minres():
    """8^3 pressure cubes, 8 spheres with jump 1e4: restarted FGMRES (restart
    20) with BFBT and a few CG steps per Z solve, against MINRES, both to a
    1e-11 residual."""
    N = 8
    p = sphere_sinkers(N, 8, 0.08, 0.01, 1e4)
    c = pkg.Context(N, pkg.default_levels(N), pkg.FP64, device=DEV)
    c.prepare(torch.from_numpy(p.eta).to(DEV), 10.0)
    b = c.load_vector(torch.from_numpy(p.fbar.ravel()).to(DEV))
    xm, itm, _ = c.solve(b, 1e-11, 20000)
    for schur, zi in (("mass", 0), ("bfbt", 20)):
        x, its, rel = c.solve_fgmres(b, 1e-11, 20000, restart=20, schur=schur, z_iters=zi)
        assert rel <= 1e-11 and its > 20
        err = float(torch.linalg.vector_norm(x - xm) / torch.linalg.vector_norm(xm))
        print(f"\n8^3 FGMRES ({schur}) {its} iterations vs MINRES {itm}: solution difference {err:.1e}")
        assert err <= 1e-7


def test_fgmres_rejects_bad_arguments(small):
    import ctypes

    _, _, c, b, _ = small
    x = torch.empty_like(b)
    sz = ctypes.c_size_t()
    lib = pkg.lib()
    assert lib.agca_fgmres_workspace_size(c._h, 0, ctypes.byref(sz)) == 1
    assert lib.agca_fgmres_workspace_size(c._h, 10, ctypes.byref(sz)) == 0
    work = torch.empty(int(sz.value), dtype=torch.uint8, device=DEV)
    its, rel = ctypes.c_int(), ctypes.c_double()
    args = (ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()))
    # too small a workspace, an unknown Schur approximation
    assert lib.agca_solve_fgmres(c._h, *args, 1e-8, 100, 10, 0, 0, ctypes.c_void_p(work.data_ptr()), 1024,
                                 ctypes.byref(its), ctypes.byref(rel)) == 2
    assert lib.agca_solve_fgmres(c._h, *args, 1e-8, 100, 10, 2, 0, ctypes.c_void_p(work.data_ptr()), sz.value,
                                 ctypes.byref(its), ctypes.byref(rel)) == 1
