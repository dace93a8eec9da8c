"""Pins of oracle.pointwise (rows of the finest operator assembled from the
elements around one vertex, Eq. 2.3) and of the viscosity-weighted lumped
pressure mass, against the oracle's global assembled matrices and closed forms.

oracle.pointwise is the only reference of the GPU apply checks at sizes where
the global sparse matrices do not fit, so it is pinned here, at every vertex
of small grids (corner, edge, face and interior vertices), against the rows of
the globally assembled operator A_L of the same field and vector.
"""
import os

import numpy as np
import pytest

from oracle import agca as oagca
from oracle import fem
from oracle.mesh import Mesh, children
from oracle.pointwise import fine_rows

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _jump_and_random_field(N, seed):
    """Per-element viscosity: a lognormal random field times a 1e4 jump on a
    grid-unaligned box, so that every element of a vertex star differs."""
    m = Mesh(2 * N)
    rng = np.random.default_rng(seed)
    eta = np.exp(rng.normal(0.0, 1.0, m.ne))
    c = m.centroids
    inside = (np.abs(c - 0.43) < 0.21).all(axis=1)
    eta[inside] *= 1e4
    return m, eta


@pytest.mark.parametrize("N", [2, 4])
def test_fine_rows_equal_rows_of_global_operator(N):
    m, eta = _jump_and_random_field(N, 11 + N)
    H = oagca.Hierarchy(N, 2, eta, 10.0)
    V = m.nv
    x = np.random.default_rng(5).uniform(-1, 1, 3 * V)
    ref = (H.A[2] @ (x * H.mask[2])).reshape(3, V).T          # rows of the masked global operator
    got = fine_rows(N, eta, x, np.arange(V))                   # boundary entries of x ignored inside
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-13 * scale
    # the check covers every kind of vertex: corners, edges and faces of the
    # boundary (rows zero) and interior vertices next to the boundary
    ijk = np.stack([np.arange(V) % (2 * N + 1), (np.arange(V) // (2 * N + 1)) % (2 * N + 1),
                    np.arange(V) // (2 * N + 1) ** 2], axis=1)
    on_bnd = ((ijk == 0) | (ijk == 2 * N)).sum(axis=1)
    assert set(on_bnd.tolist()) == {0, 1, 2, 3}
    assert np.abs(got[on_bnd > 0]).max() == 0.0
    assert np.abs(got[on_bnd == 0]).min() > 0.0


def test_fine_rows_see_boundary_values_only_through_the_mask():
    """Dirichlet: changing x on boundary vertices changes no row."""
    N = 2
    m, eta = _jump_and_random_field(N, 3)
    x = np.random.default_rng(8).uniform(-1, 1, 3 * m.nv)
    x2 = x.copy()
    bnd = np.nonzero(~m.interior)[0]
    for c in range(3):
        x2[c * m.nv + bnd] = 7.0
    verts = np.arange(m.nv)
    assert np.array_equal(fine_rows(N, eta, x, verts), fine_rows(N, eta, x2, verts))


def test_pressure_mass_weight_is_mean_of_inverse_viscosity():
    """w_T = mean of 1/eta over the 8 velocity children of pressure element T:
    with eta = a on 4 children and b on the other 4, w = (1/a + 1/b) / 2
    (neither 1/mean(eta) = 2/(a + b) nor mean(eta))."""
    pm, vm = Mesh(2), Mesh(4)
    ch = children(pm, vm)
    a, b = 3.0, 1e-2
    eta = np.empty(vm.ne)
    eta[ch[:, :4].ravel()] = a
    eta[ch[:, 4:].ravel()] = b
    M = fem.pressure_mass_lumped(pm, eta, ch)
    w = 0.5 * (1.0 / a + 1.0 / b)
    assert abs(M.sum() - w) <= 1e-13 * w                    # total volume 1
    M1 = fem.pressure_mass_lumped(pm, np.ones(vm.ne), ch)
    assert np.allclose(M, w * M1, rtol=1e-14, atol=0)
    # per-element two-valued weights: sum_T w_T |T| with w_T from the closed form
    rng = np.random.default_rng(2)
    aa, bb = np.exp(rng.normal(size=pm.ne)), np.exp(rng.normal(size=pm.ne))
    eta[ch[:, :4]] = aa[:, None]
    eta[ch[:, 4:]] = bb[:, None]
    M = fem.pressure_mass_lumped(pm, eta, ch)
    wT = 0.5 * (1.0 / aa + 1.0 / bb)
    assert abs(M.sum() - (wT * pm.volumes).sum()) <= 1e-13 * M.sum()


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_paper_sizes_and_memory_model():
    """Section 4's problem size and Section 5's memory model (Eqs. 5.1-5.8)
    from this grid's own counts."""
    g = _golden("paper_sizes.txt")
    # 48 macro elements (the 2^3-cube Kuhn grid) refined 5 times: pressure on
    # 64 cubes per axis, velocity on 128 (P1-iso-P2)
    assert 6 * 2 ** 3 == g["macro_elements_section4"]
    N = 2 * 2 ** 5
    dofs = 3 * (2 * N + 1) ** 3 + (N + 1) ** 3
    assert round(dofs / 1e5) / 10 == g["dofs_section4"] / 1e6
    # Eq. 5.1: 8 times more vertices per refinement, velocity DoFs 3 per vertex
    c_u = 1.0 - 1.0 / (3 * 8)
    assert abs(c_u - g["c_u"]) < 0.01
    assert abs(dofs - 3 * (2 * N + 1) ** 3 - (1 - c_u) * dofs) < 0.01 * dofs
    # Eq. 5.4: the Galerkin matrix on a grid with 1/8 of the vertices
    assert abs(g["mem_A"] / 8 - g["mem_gca_sparse"]) < 0.05
    # Eq. 5.6: 3 components x 16 entries x 6 elements per vertex x 1/8
    assert abs(3 * 16 * 6 / 8 * c_u - g["mem_agca_elementwise"]) < 0.02 * g["mem_agca_elementwise"]
    # Eq. 5.8: 3 components x 15 stencil entries x 1/8
    assert abs(3 * 15 / 8 * c_u - g["mem_agca_stencil"]) < 0.01 * g["mem_agca_stencil"]
