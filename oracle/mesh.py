"""Kuhn tetrahedral meshes of the unit cube and their multigrid relations.

Section 2 (Eq. 2.2) builds the grid by uniform refinement of macro elements;
here the macro mesh is the coarsest Kuhn cube grid and every refinement halves
the cube size, which refines each tetrahedron into eight (Fig. 2).

Everything geometric is derived from vertex coordinates: barycentric
coordinates and gradients by inverting the 4x4 matrix [1; x], volumes from
its determinant, parents by locating child centroids, interpolation weights
by evaluating coarse barycentric coordinates at fine vertices.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


class Mesh:
    """Kuhn mesh with n cubes per axis on [0,1]^3.

    vertex id = i + (n+1)*(j + (n+1)*k); element id = 6*cube_id + t.
    tets[e] lists the element's vertices in the order v0 (cube origin),
    v1 = v0 + e_p0, v2 = v1 + e_p1, v3 = v0 + (1,1,1).
    """

    def __init__(self, n: int):
        self.n = n
        self.h = 1.0 / n
        m = n + 1
        self.nv = m ** 3
        self.ne = 6 * n ** 3
        g = np.arange(m)
        K, J, I = np.meshgrid(g, g, g, indexing="ij")
        self.coords = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1) * self.h
        self.ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
        c = np.arange(n)
        K, J, I = np.meshgrid(c, c, c, indexing="ij")
        org = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)  # cube origins
        tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
        for t, p in enumerate(PERMS):
            v = org.copy()
            tets[:, t, 0] = self.vid(v)
            for a in range(3):
                v = v.copy()
                v[:, p[a]] += 1
                tets[:, t, a + 1] = self.vid(v)
        self.tets = tets.reshape(-1, 4)
        on_bd = (self.ijk == 0) | (self.ijk == n)
        self.interior = ~on_bd.any(axis=1)

    def vid(self, ijk):
        m = self.n + 1
        ijk = np.asarray(ijk)
        return ijk[..., 0] + m * (ijk[..., 1] + m * ijk[..., 2])

    @functools.cached_property
    def bary_inverse(self):
        """(E,4,4): rows a give lambda_a(x) = Minv[a,0] + Minv[a,1:4].x."""
        X = self.coords[self.tets]                       # (E,4,3)
        M = np.ones((self.ne, 4, 4))
        M[:, 1:, :] = np.transpose(X, (0, 2, 1))
        return np.linalg.inv(M)

    @functools.cached_property
    def grads(self):
        """(E,4,3) gradients of the element's barycentric functions."""
        return self.bary_inverse[:, :, 1:].copy()

    @functools.cached_property
    def volumes(self):
        X = self.coords[self.tets]
        M = np.ones((self.ne, 4, 4))
        M[:, 1:, :] = np.transpose(X, (0, 2, 1))
        return np.abs(np.linalg.det(M)) / 6.0

    @functools.cached_property
    def centroids(self):
        return self.coords[self.tets].mean(axis=1)

    def barycentric(self, elems, x):
        """Barycentric coordinates of points x (P,3) in elements elems (P,)."""
        Minv = self.bary_inverse[elems]
        return Minv[:, :, 0] + np.einsum("pai,pi->pa", Minv[:, :, 1:], x)

    def locate(self, x, tol=1e-12):
        """Element containing each point (first match in element-id order)."""
        x = np.atleast_2d(x)
        cube = np.clip(np.floor(x * self.n + 1e-9).astype(np.int64), 0, self.n - 1)
        # a point on a cube face may belong to the neighbouring cube as well;
        # try the 8 candidate cubes around it
        best = np.full(len(x), -1, dtype=np.int64)
        for dz in (0, -1):
            for dy in (0, -1):
                for dx in (0, -1):
                    cc = cube + np.array([dx, dy, dz])
                    ok = (cc >= 0).all(axis=1) & (cc < self.n).all(axis=1)
                    cid = cc[:, 0] + self.n * (cc[:, 1] + self.n * cc[:, 2])
                    for t in range(6):
                        e = 6 * cid + t
                        sel = ok & (best < 0)
                        if not sel.any():
                            continue
                        lam = self.barycentric(e[sel], x[sel])
                        inside = (lam >= -tol).all(axis=1)
                        idx = np.nonzero(sel)[0][inside]
                        best[idx] = e[sel][inside]
        assert (best >= 0).all(), "point outside the mesh"
        return best


def parents(coarse: Mesh, fine: Mesh) -> np.ndarray:
    """Parent coarse element of every fine element, by centroid containment."""
    assert fine.n == 2 * coarse.n
    return coarse.locate(fine.centroids)


def children_brute(coarse: Mesh, fine: Mesh) -> np.ndarray:
    """(E_coarse, 8) children of each coarse element, ascending fine element
    id, by locating every fine centroid in the coarse mesh."""
    par = parents(coarse, fine)
    order = np.argsort(par, kind="stable")
    ch = order.reshape(coarse.ne, 8)
    assert (par[ch] == np.arange(coarse.ne)[:, None]).all()
    return ch


@functools.lru_cache(maxsize=None)
def child_table() -> np.ndarray:
    """(6, 8, 4): for a parent of Kuhn type t, its children as (ox, oy, oz, t')
    = sub-cube offset and child type, ascending child element id.  Found by
    centroid containment on the one-cube mesh refined once."""
    ch = children_brute(Mesh(1), Mesh(2))               # (6, 8) fine ids
    t_child = ch % 6
    cube = ch // 6
    ox, oy, oz = cube % 2, (cube // 2) % 2, cube // 4
    return np.stack([ox, oy, oz, t_child], axis=-1)


def children(coarse: Mesh, fine: Mesh) -> np.ndarray:
    """(E_coarse, 8) children of each coarse element, ascending fine element
    id: the one-cube containment table translated to every coarse cube (the
    refinement is translation invariant)."""
    assert fine.n == 2 * coarse.n
    return children_n(coarse.n)


def children_n(n: int) -> np.ndarray:
    """children() for a coarse mesh of n cubes per axis (no mesh needed)."""
    tab = child_table()
    e = np.arange(6 * n ** 3)
    t = e % 6
    cid = e // 6
    I, J, K = cid % n, (cid // n) % n, cid // (n * n)
    o = tab[t]                                           # (E,8,4)
    fi = 2 * I[:, None] + o[:, :, 0]
    fj = 2 * J[:, None] + o[:, :, 1]
    fk = 2 * K[:, None] + o[:, :, 2]
    nf = 2 * n
    return 6 * (fi + nf * (fj + nf * fk)) + o[:, :, 3]


def prolongation(coarse: Mesh, fine: Mesh) -> sp.csr_matrix:
    """Scalar linear interpolation P (V_fine x V_coarse): the coarse P1
    function evaluated at fine vertices (Sec. 2.1, canonical embedding)."""
    e = coarse.locate(fine.coords)
    lam = coarse.barycentric(e, fine.coords)
    rows = np.repeat(np.arange(fine.nv), 4)
    cols = coarse.tets[e].ravel()
    vals = lam.ravel()
    keep = np.abs(vals) > 1e-14
    P = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(fine.nv, coarse.nv))
    return P.tocsr()


def local_interpolation(coarse: Mesh, fine: Mesh, ch: np.ndarray, elems=None) -> np.ndarray:
    """Local interpolation matrices of Eq. 2.4: p[e, k, i, j] = lambda_j of the
    parent e at vertex i of its k-th child (shape (E', 8, 4, 4))."""
    if elems is None:
        elems = np.arange(coarse.ne)
    kids = ch[elems]                                     # (E',8)
    pts = fine.coords[fine.tets[kids]]                   # (E',8,4,3)
    par = np.repeat(elems, 32)
    lam = coarse.barycentric(par, pts.reshape(-1, 3))
    return lam.reshape(len(elems), 8, 4, 4)
