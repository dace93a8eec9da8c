"""Pins of the oracle's Stokes discretization and solvers: a manufactured
solution's convergence orders (P1-iso-P2 / P1 pair of Eq. 3.3, Bercovier and
Pironneau), MINRES against a sparse direct solve, and the adjoint gradient
against central finite differences."""
import numpy as np
import pytest
import sympy as s

from oracle import agca, fem, stokes
from oracle.mesh import Mesh
from synth import cube_sinker, sphere_sinkers

_A, _B = 0.5854101966249685, 0.1381966011250105


def _manufactured():
    x, y, z = s.symbols("x y z")
    phi = s.sin(s.pi * x) ** 2 * s.sin(s.pi * y) ** 2 * s.sin(s.pi * z)
    u = [s.diff(phi, y), -s.diff(phi, x), s.Integer(0)]
    p = s.cos(s.pi * x) * s.cos(s.pi * y) * s.cos(s.pi * z)
    eta = 1 + s.sin(2 * s.pi * x) / 2
    X = [x, y, z]
    grad = [[s.diff(u[i], X[j]) for j in range(3)] for i in range(3)]
    eps = [[(grad[i][j] + grad[j][i]) / 2 for j in range(3)] for i in range(3)]
    f = [-sum(s.diff(2 * eta * eps[i][j], X[j]) for j in range(3)) + s.diff(p, X[i]) for i in range(3)]
    lam = lambda e: s.lambdify((x, y, z), e, "numpy")
    return ([lam(c) for c in u], [[lam(grad[i][j]) for j in range(3)] for i in range(3)],
            lam(p), lam(eta), [lam(c) for c in f])


def _qpoints(m):
    X = m.coords[m.tets]
    return _B * X.sum(axis=1, keepdims=True) + (_A - _B) * X   # (E,4,3)


def _ev(fn, P):
    v = fn(P[..., 0], P[..., 1], P[..., 2])
    return np.broadcast_to(v, P.shape[:-1]).astype(float)


def _errors(N, man):
    u_fn, gu_fn, p_fn, eta_fn, f_fn = man
    L = 2
    vm = Mesh(2 * N)
    Q = _qpoints(vm)
    eta = _ev(eta_fn, Q).mean(axis=1)
    H = agca.Hierarchy(N, L, eta, 10.0)
    S = stokes.Stokes(H)
    b = np.zeros(S.nu_ + S.np_)
    b[:S.nu_] = fem.load_vector_quadrature(vm, lambda P: np.stack([_ev(f, P) for f in f_fn], axis=1))
    x = S.direct(b)
    u, p = S.split(x)
    w = vm.volumes[:, None] / 4.0
    U = np.stack([u[c * vm.nv + vm.tets] for c in range(3)], axis=-1)    # (E,4,3)
    phi = np.full((4, 4), _B)
    np.fill_diagonal(phi, _A)
    Uq = np.einsum("qa,eac->eqc", phi, U)
    ue = np.stack([_ev(f, Q) for f in u_fn], axis=-1)
    l2u = np.sqrt((w[..., None] * (ue - Uq) ** 2).sum())
    Gh = np.einsum("eac,eaj->ecj", U, vm.grads)                          # (E,3,3)
    Ge = np.stack([np.stack([_ev(gu_fn[i][j], Q) for j in range(3)], -1) for i in range(3)], -2)
    h1u = np.sqrt((w[..., None, None] * (Ge - Gh[:, None]) ** 2).sum())
    pm = S.pm
    Qp = _qpoints(pm)
    Pq = np.einsum("qa,ea->eq", phi, p[pm.tets])
    diff = _ev(p_fn, Qp) - Pq
    wp = pm.volumes[:, None] / 4.0
    diff = diff - (wp * diff).sum() / wp.sum()
    l2p = np.sqrt((wp * diff ** 2).sum())
    return l2u, h1u, l2p


def test_manufactured_solution_orders():
    man = _manufactured()
    e4 = _errors(4, man)
    e8 = _errors(8, man)
    rates = [np.log2(a / b) for a, b in zip(e4, e8)]
    # L2 velocity O(h^2), H1 velocity O(h), L2 pressure at least O(h)
    assert rates[0] > 1.8, rates
    assert 0.85 < rates[1] < 1.3, rates
    assert rates[2] > 0.9, rates


@pytest.fixture(scope="module")
def stokes_small():
    p = sphere_sinkers(4, n_sinkers=2, radius=0.15, width=0.03, dr=1e4)
    H = agca.Hierarchy(4, 3, p.eta, 10.0)
    S = stokes.Stokes(H)
    return S, S.rhs(p.fbar)


def test_minres_matches_direct(stokes_small):
    S, b = stokes_small
    xd = S.direct(b)
    assert np.linalg.norm(b - S.K(xd)) <= 1e-10 * np.linalg.norm(b)
    x, its = S.solve(b, rtol=1e-12, inner_rtol=1e-13)
    assert np.linalg.norm(b - S.K(x)) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert abs(x[S.nu_:].mean()) < 1e-14 * np.abs(x[S.nu_:]).max()


def test_preconditioner_symmetric(stokes_small):
    S, b = stokes_small
    rng = np.random.default_rng(3)
    n = len(b)
    m = np.concatenate([S.mask, np.ones(S.np_)])
    x, y = rng.normal(size=n) * m, rng.normal(size=n) * m
    x[S.nu_:] -= x[S.nu_:].mean()
    y[S.nu_:] -= y[S.nu_:].mean()
    a1, a2 = y @ S.precondition(x), x @ S.precondition(y)
    assert abs(a1 - a2) <= 1e-12 * abs(a1)


def test_adjoint_gradient_matches_finite_differences():
    p = sphere_sinkers(2, n_sinkers=1, radius=0.2, width=0.05, dr=1e2)
    theta = np.log(p.eta)
    rng = np.random.default_rng(4)

    def solve(th):
        H = agca.Hierarchy(2, 2, np.exp(th), 10.0)
        S = stokes.Stokes(H)
        return S, S.direct(S.rhs(p.fbar))

    S, x = solve(theta)
    u_obs = rng.normal(size=S.nu_) * S.mask * 1e-3
    J = lambda xx: 0.5 * np.sum((xx[:S.nu_] - u_obs) ** 2)
    g = S.adjoint_gradient(x, u_obs)
    for _ in range(4):
        d = rng.normal(size=theta.shape)
        eps = 1e-4
        Jp = J(solve(theta + eps * d)[1])
        Jm = J(solve(theta - eps * d)[1])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd), (fd, g @ d)


@pytest.mark.slow
def test_cube_sinker_solve_reaches_tolerance():
    p = cube_sinker(8)
    H = agca.Hierarchy(8, 3, p.eta, 10.0)
    S = stokes.Stokes(H)
    b = S.rhs(p.fbar)
    x, its = S.solve(b, 1e-8)
    assert np.linalg.norm(b - S.K(x)) <= 1e-8 * np.linalg.norm(b)
    xd = S.direct(b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
