"""Pins of the oracle's AGCA hierarchy (Sec. 2.2-2.3, Eqs. 2.5-2.9) and of its
smoother and V-cycle against brute force, closed forms and invariants."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import agca, fem
from oracle.mesh import Mesh
from synth import cube_sinker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_splitmix64_published_values():
    want = [int(r[0], 16) for r in _golden_rows("splitmix64_seed0.txt")]
    got = [int(v) for v in agca.splitmix64(np.arange(3))]
    assert got == want
    v = agca.start_vector(1000)
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.1


def test_flag_counts_cube_sinker():
    p = cube_sinker(16)
    _, _, _, flags = agca.flag_hierarchy(16, 4, p.eta, 10.0)
    want = {int(r[0]): (int(r[1]), int(r[2])) for r in _golden_rows("flag_counts.txt")}
    for l in (1, 2, 3):
        n = 32 >> (4 - l)
        assert (int(flags[l].sum()), flags[l].size) == want[n]


def test_aligned_sinker_no_flags_and_agca_equals_dca():
    """A jump aligned with every grid is represented exactly by DCA (Sec. 4.1,
    Fig. 8 eta_1): nothing is flagged and AGCA reduces to DCA."""
    p = cube_sinker(8, lo=0.25, hi=0.75)
    H = agca.Hierarchy(8, 3, p.eta, 10.0, build_operators=False)
    assert all(not H.flags[l].any() for l in (1, 2))
    # and for this field the DCA means are exactly the Galerkin matrices
    Hall = agca.Hierarchy(8, 3, p.eta, 0.5, build_operators=False)
    for l in (1, 2):
        dca = fem.element_matrices(Hall.mesh[l], Hall.mean[l])
        assert np.allclose(Hall.gca[l], dca, rtol=1e-13, atol=1e-13 * np.abs(dca).max())


def test_dca_equals_gca_for_constant_viscosity():
    """Sec. 2.1: with constant coefficients DCA and GCA coincide."""
    for N, L in ((2, 2), (4, 3)):
        m = Mesh(2 * N)
        H = agca.Hierarchy(N, L, np.full(m.ne, 3.7), 0.5, build_operators=False)
        for l in range(1, L):
            dca = fem.element_matrices(H.mesh[l], np.full(H.mesh[l].ne, 3.7))
            assert np.abs(H.gca[l] - dca).max() <= 1e-13 * np.abs(dca).max()


@pytest.mark.parametrize("N,L", [(2, 2), (4, 2), (4, 3)])
def test_elementwise_galerkin_equals_global_triple_product(N, L):
    """Eq. 2.6: with every coarse element flagged the element-wise assembly
    equals the global sparse product P^T A_{l+1} P (masked to Dirichlet)."""
    rng = np.random.default_rng(10 + N)
    m = Mesh(2 * N)
    eta = np.exp(rng.uniform(-4, 4, m.ne))
    H = agca.Hierarchy(N, L, eta, 0.5)
    for l in range(1, L):
        assert H.flags[l].all()
        brute = (H.P[l].T @ H.A[l + 1] @ H.P[l]).toarray()
        got = H.A[l].toarray()
        assert np.abs(got - brute).max() <= 1e-13 * np.abs(brute).max()


def test_viscosity_hierarchy_invariants():
    rng = np.random.default_rng(5)
    m = Mesh(8)
    eta = np.exp(rng.uniform(-3, 3, m.ne))
    mean, mx, mn, flags = agca.flag_hierarchy(4, 3, eta, 10.0)
    H = agca.Hierarchy(4, 3, eta, 10.0, build_operators=False)
    for l in (1, 2):
        kids = H.ch[l]
        plain = H.mean[l + 1][kids].mean(axis=1)
        assert np.allclose(mean[l], plain, rtol=1e-15)
        assert (mx[l] >= mean[l]).all() and (mean[l] >= mn[l]).all()
        assert (mean[l] == H.mean[l]).all() and (flags[l] == H.flags[l]).all()
    # a flagged child implies a flagged parent
    kids = H.ch[1]
    assert (H.flags[1][H.flags[2][kids].any(axis=1)]).all()


@pytest.fixture(scope="module")
def hier_small():
    rng = np.random.default_rng(7)
    m = Mesh(8)
    eta = np.exp(rng.uniform(-3, 3, m.ne))
    return agca.Hierarchy(4, 3, eta, 10.0)


def test_agca_operator_spd(hier_small):
    H = hier_small
    for l in (1, 2, 3):
        A = H.A[l]
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
        idx = np.nonzero(H.mask[l])[0]
        if len(idx) < 800:
            w = np.linalg.eigvalsh(A[idx][:, idx].toarray())
            assert w.min() > 0


def test_power_iteration_bounds(hier_small):
    """lambda_hat is a Rayleigh quotient of the pencil (A, D): never above its
    largest eigenvalue, and close to it after the fixed iteration count."""
    H = hier_small
    for l in (2,):
        idx = np.nonzero(H.mask[l])[0]
        A = H.A[l][idx][:, idx].toarray()
        D = H.D[l][idx]
        lmax = sla.eigh(A, np.diag(D), eigvals_only=True)[-1]
        assert H.lam[l] <= lmax * (1 + 1e-12)
        assert H.lam[l] >= 0.9 * lmax


def test_chebyshev_error_polynomial(hier_small):
    """The smoother's error propagation equals the scaled Chebyshev polynomial
    T_k((theta - D^-1 A)/delta) / T_k(theta/delta) of degree k."""
    H = hier_small
    l = 2
    idx = np.nonzero(H.mask[l])[0]
    A = H.A[l][idx][:, idx].toarray()
    d = H.D[l][idx]
    S = A / np.sqrt(np.outer(d, d))
    w, Q = np.linalg.eigh(S)
    a, b = H.cheb_lo * H.lam[l], H.cheb_hi * H.lam[l]
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    T2 = lambda t: 2 * t * t - 1
    q = T2((theta - w) / delta) / T2(theta / delta)
    E_want = (Q * q) @ Q.T                                 # in the D^1/2 basis
    n = 3 * H.mesh[l].nv
    E_got = np.zeros((len(idx), len(idx)))
    for j, col in enumerate(idx):
        e0 = np.zeros(n)
        e0[col] = 1.0
        # error after smoothing A x = A e0 from x = 0: e = e0 - x
        x = H.chebyshev(l, H.A[l] @ e0, np.zeros(n))
        E_got[:, j] = (e0 - x)[idx]
    sd = np.sqrt(d)
    E_got = sd[:, None] * E_got / sd[None, :]
    assert np.abs(E_got - E_want).max() < 1e-11


def test_vcycle_symmetric_positive_contracting(hier_small):
    H = hier_small
    n = 3 * H.mesh[3].nv
    rng = np.random.default_rng(8)
    x, y = rng.normal(size=n) * H.mask[3], rng.normal(size=n) * H.mask[3]
    Vx, Vy = H.vcycle(x), H.vcycle(y)
    assert abs(y @ Vx - x @ Vy) <= 1e-12 * abs(y @ Vx)
    assert x @ Vx > 0 and y @ Vy > 0
    # error propagation I - V A contracts in the energy norm
    e = rng.normal(size=n) * H.mask[3]
    for _ in range(3):
        e = e - H.vcycle(H.A[3] @ e)
    e2 = e - H.vcycle(H.A[3] @ e)
    assert np.sqrt(e2 @ (H.A[3] @ e2)) < 0.5 * np.sqrt(e @ (H.A[3] @ e))


def test_coarse_solve_exact(hier_small):
    H = hier_small
    n = 3 * H.mesh[1].nv
    b = np.random.default_rng(9).normal(size=n) * H.mask[1]
    x = H.coarse_solve(b)
    assert np.abs(H.A[1] @ x - b).max() < 1e-10 * np.abs(b).max()
