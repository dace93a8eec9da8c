"""Rows of the finest-level operators at sampled vertices, for checks at sizes
where the global sparse matrices of the oracle do not fit.

Each row is assembled from the elements around the vertex (Eq. 2.3): the 24
Kuhn tetrahedra of the 8 cubes sharing the vertex, with geometry computed
from vertex coordinates by the same barycentric inversion as oracle.mesh.
"""
from __future__ import annotations

import numpy as np

from .mesh import PERMS


def _elements_around(n, i, j, k):
    """(element id, local vertex ids (4,3) integer coords) of tets containing
    vertex (i, j, k) on an n-cube Kuhn grid."""
    out = []
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                c = np.array([i - ox, j - oy, k - oz])
                if (c < 0).any() or (c >= n).any():
                    continue
                cid = c[0] + n * (c[1] + n * c[2])
                for t, p in enumerate(PERMS):
                    verts = [c.copy()]
                    v = c.copy()
                    for a in range(3):
                        v = v.copy()
                        v[p[a]] += 1
                        verts.append(v)
                    verts = np.array(verts)
                    if any((vv == [i, j, k]).all() for vv in verts):
                        out.append((6 * cid + t, verts))
    return out


def _element_matrix(verts_int, h, eta):
    X = verts_int * h
    M = np.ones((4, 4))
    M[1:, :] = X.T
    Minv = np.linalg.inv(M)
    G = Minv[:, 1:]
    vol = abs(np.linalg.det(M)) / 6.0
    A = np.zeros((3, 4, 3, 4))
    gg = G @ G.T
    for c in range(3):
        A[c, :, c, :] += gg
    A += np.einsum("ad,bc->cadb", G, G)
    return (eta * vol * A).reshape(12, 12)


def fine_rows(N: int, eta: np.ndarray, x: np.ndarray, vertices) -> np.ndarray:
    """(A_L x) at the given vertex ids, shape (len(vertices), 3); boundary
    vertices give 0 and boundary entries of x are ignored (Dirichlet)."""
    n = 2 * N
    m = n + 1
    V = m ** 3
    h = 1.0 / n

    def interior(ijk):
        return (ijk > 0).all() and (ijk < n).all()

    out = np.zeros((len(vertices), 3))
    for r, v in enumerate(vertices):
        i, j, k = v % m, (v // m) % m, v // (m * m)
        if not interior(np.array([i, j, k])):
            continue
        for e, verts in _elements_around(n, i, j, k):
            A = _element_matrix(verts, h, eta[e])
            vid = verts[:, 0] + m * (verts[:, 1] + m * verts[:, 2])
            xe = np.zeros(12)
            for c in range(3):
                for a in range(4):
                    if interior(verts[a]):
                        xe[c * 4 + a] = x[c * V + vid[a]]
            ye = A @ xe
            a_self = [a for a in range(4) if vid[a] == v][0]
            for c in range(3):
                out[r, c] += ye[c * 4 + a_self]
    return out
