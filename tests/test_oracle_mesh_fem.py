"""Pins of the oracle's geometry and finite-element pieces against closed forms
and invariants (Sec. 2, Eqs. 2.2-2.4, Eqs. 3.3-3.5)."""
import numpy as np
import pytest

from oracle import fem
from oracle.mesh import Mesh, children, children_brute, child_table, local_interpolation, prolongation


@pytest.mark.parametrize("n", [1, 2, 3])
def test_geometry_closed_forms(n):
    m = Mesh(n)
    h = 1.0 / n
    assert np.allclose(m.volumes, h ** 3 / 6, rtol=0, atol=1e-15)
    assert abs(m.volumes.sum() - 1.0) < 1e-13
    # barycentric functions: lambda_a(x_b) = delta_ab, gradients sum to zero
    lam = m.barycentric(np.repeat(np.arange(m.ne), 4), m.coords[m.tets].reshape(-1, 3))
    assert np.allclose(lam.reshape(m.ne, 4, 4), np.eye(4)[None], atol=1e-13)
    assert np.abs(m.grads.sum(axis=1)).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3])
def test_children_structural_equals_containment(n):
    c, f = Mesh(n), Mesh(2 * n)
    assert (children(c, f) == children_brute(c, f)).all()


def test_child_table_structure():
    tab = child_table()
    for t in range(6):
        offs = [tuple(r[:3]) for r in tab[t]]
        # two children in the diagonal sub-cubes, six from the others
        assert offs.count((0, 0, 0)) == 1 and offs.count((1, 1, 1)) == 1
    c, f = Mesh(2), Mesh(4)
    ch = children(c, f)
    assert np.allclose(f.volumes[ch].sum(axis=1), c.volumes)
    p = local_interpolation(c, f, ch)
    # child vertices lie in the parent; weights are 0, 1/2 or 1
    assert (p > -1e-13).all() and np.allclose(p.sum(axis=-1), 1.0)
    assert np.allclose(np.round(2 * p), 2 * p, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_prolongation_reproduces_linears(n):
    c, f = Mesh(n), Mesh(2 * n)
    P = prolongation(c, f)
    rng = np.random.default_rng(0)
    a, g = rng.normal(), rng.normal(size=3)
    assert np.allclose(P @ (a + c.coords @ g), a + f.coords @ g, atol=1e-13)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)
    # even fine vertices copy, odd ones average two coarse vertices (Kuhn edges)
    nnz = np.diff(P.indptr)
    assert set(np.unique(nnz)) <= {1, 2}


def _linear_field_dofs(m, G, c0):
    """Local nodal values (E,12) of u(x) = G x + c0, local index c*4 + a."""
    X = m.coords[m.tets]                                  # (E,4,3)
    U = X @ G.T + c0                                      # (E,4,3)
    return np.transpose(U, (0, 2, 1)).reshape(m.ne, 12)


def test_element_matrix_bilinear_form_closed_form():
    """The 12 local DoFs span exactly the linear fields, so the element matrix
    is fixed by its bilinear form on them: for u = G1 x + c1, v = G2 x + c2,
    v^T A_e u = 2 eta |T| sym(G1) : sym(G2)  (Eq. 3.5 with constant strain)."""
    m = Mesh(2)
    rng = np.random.default_rng(1)
    eta = rng.uniform(0.1, 10.0, m.ne)
    A = fem.element_matrices(m, eta)
    for _ in range(4):
        G1, G2 = rng.normal(size=(3, 3)), rng.normal(size=(3, 3))
        u = _linear_field_dofs(m, G1, rng.normal(size=3))
        v = _linear_field_dofs(m, G2, rng.normal(size=3))
        got = np.einsum("ei,eij,ej->e", v, A, u)
        S1, S2 = 0.5 * (G1 + G1.T), 0.5 * (G2 + G2.T)
        want = 2.0 * eta * m.volumes * (S1 * S2).sum()
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


def test_element_matrix_invariants():
    m = Mesh(1)
    A = fem.element_matrices(m, np.ones(m.ne))
    assert np.abs(A - A.transpose(0, 2, 1)).max() == 0.0
    X = m.coords[m.tets]
    modes = []
    for c in range(3):
        r = np.zeros((m.ne, 3, 4))
        r[:, c, :] = 1.0
        modes.append(r.reshape(m.ne, 12))
    for ax in range(3):
        w = np.zeros(3)
        w[ax] = 1.0
        modes.append(np.transpose(np.cross(w, X), (0, 2, 1)).reshape(m.ne, 12))
    for r in modes:   # translations and rotations are strain free
        assert np.abs(np.einsum("eij,ej->ei", A, r)).max() < 1e-14
    for e in range(6):
        assert np.linalg.matrix_rank(A[e]) == 6
        assert (np.abs(A[e]) > 1e-12).sum() == 54


def test_global_energy_of_linear_field():
    m = Mesh(3)
    rng = np.random.default_rng(2)
    eta = rng.uniform(0.5, 2.0, m.ne)
    A = fem.assemble(m, fem.element_matrices(m, eta))
    G = rng.normal(size=(3, 3))
    U = m.coords @ G.T
    u = U.T.ravel()                                       # SoA
    S = 0.5 * (G + G.T)
    assert np.isclose(u @ (A @ u), 2.0 * (S * S).sum() * (eta * m.volumes).sum(), rtol=1e-12)
    assert abs((A - A.T)).max() < 1e-15


def test_divergence_closed_forms():
    """D u for u = G x: int psi_k tr(G) = tr(G) * (sum_{T ni k} |T| / 4)."""
    from oracle.mesh import parents
    pm, vm = Mesh(2), Mesh(4)
    par = parents(pm, vm)
    D = fem.divergence(pm, vm, par)
    rng = np.random.default_rng(3)
    G = rng.normal(size=(3, 3))
    u = (vm.coords @ G.T).T.ravel()
    mass = np.zeros(pm.nv)
    np.add.at(mass, pm.tets.ravel(), np.repeat(pm.volumes / 4, 4))
    assert np.allclose(D @ u, np.trace(G) * mass, rtol=1e-12, atol=1e-15)
    # constants are in the kernel of B^T on interior velocity DoFs
    mask = fem.velocity_mask(vm)
    assert np.abs((D.T @ np.ones(pm.nv)) * mask).max() < 1e-14


def test_load_vector_and_pressure_mass():
    m = Mesh(2)
    fbar = np.zeros((3, m.ne))
    fbar[2] = 1.0
    b = fem.load_vector(m, fbar)
    # interior vertices: the integral of the hat function = h^3 on a Kuhn grid
    iv = np.nonzero(m.interior)[0]
    assert np.allclose(b[2 * m.nv + iv], m.h ** 3)
    assert np.abs(b[:2 * m.nv]).max() == 0.0
    pm = Mesh(1)
    ch = children(pm, m)
    M = fem.pressure_mass_lumped(pm, np.ones(m.ne), ch)
    assert abs(M.sum() - 1.0) < 1e-14
