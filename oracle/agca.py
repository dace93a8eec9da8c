"""Adaptive Galerkin coarse-grid approximation (Section 2) on Kuhn meshes.

Levels l = 1 (coarsest) .. L (finest); level l has n_L / 2^(L-l) cubes per
axis.  Level L is always matrix-free with the element-mean viscosity; a
coarse element is Galerkin-coarsened when the viscosities of the finest
elements it covers vary by more than the threshold:

  flag(e) := max_e > nu * min_e       (element-wise form of Eq. 2.8)

Flagged elements store A_e^GCA = sum_k (I3 x p_k)^T C_k (I3 x p_k) over their
8 children (Eqs. 2.6-2.7, Eq. B.2), where C_k is the child's finest matrix,
its stored Galerkin matrix, or its direct (DCA, Eq. 2.5) matrix built from
the arithmetic mean of the child's viscosity (or its harmonic or geometric
mean: the P0 projections of Sec. 3.2).  Unflagged elements use DCA.
gradient_flags gives the paper's own flag rule (Eq. 2.8: gradient norm of
the P1-interpolated viscosity above nu), with coarse elements in the role of
macro elements.
The level operator is the heterogeneous sum of Eq. 2.9.

The V-cycle uses Chebyshev smoothing on D^-1 A (Section 4, degree 2 by
default) with an interval [lo, hi] * lambda_hat, lambda_hat from a fixed
number of power iterations started from a splitmix64 vector, and an exact
(Cholesky) coarsest-grid solve.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem
from .mesh import Mesh, children, children_n, local_interpolation, prolongation

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(idx: np.ndarray, seed: int = 0) -> np.ndarray:
    """SplitMix64 output for counter values idx (Steele, Lea, Flood 2014)."""
    z = np.uint64(seed) + (idx.astype(np.uint64) + np.uint64(1)) * _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def start_vector(n: int) -> np.ndarray:
    """Power-iteration start vector: splitmix64(i) mapped to [-1, 1)."""
    u = (splitmix64(np.arange(n)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return 2.0 * u - 1.0


def pairwise8(c: np.ndarray) -> np.ndarray:
    """((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)) along the last axis."""
    return ((c[..., 0] + c[..., 1]) + (c[..., 2] + c[..., 3])) + \
           ((c[..., 4] + c[..., 5]) + (c[..., 6] + c[..., 7]))


PROJECTIONS = ("arithmetic", "harmonic", "geometric")


def coarse_mean(c: np.ndarray, projection: str = "arithmetic") -> np.ndarray:
    """Piecewise-constant (P0) coefficient of a parent from its 8 children's
    values c[..., 8]: the arithmetic, harmonic or geometric mean, the three
    P0 projections of Sec. 3.2 (Fig. 6).  Sums run in the pairwise8 order."""
    if projection == "arithmetic":
        return pairwise8(c) * 0.125
    if projection == "harmonic":
        return 8.0 / pairwise8(1.0 / c)
    if projection == "geometric":
        return np.exp(pairwise8(np.log(c)) * 0.125)
    raise ValueError(f"unknown projection {projection!r}")


def gradient_norms(mesh: Mesh, eta_v: np.ndarray) -> np.ndarray:
    """Per element of mesh, the norm of the gradient of the P1 interpolant
    with nodal values eta_v (the quantity Eq. 2.8 thresholds), from the
    element's barycentric gradients."""
    g = np.einsum("ea,eai->ei", np.asarray(eta_v, dtype=np.float64)[mesh.tets], mesh.grads)
    return np.sqrt(np.einsum("ei,ei->e", g, g))


def gradient_flags(N: int, L: int, eta_v: np.ndarray, nu: float):
    """The flag rule of Eq. 2.8 with the level-l element in the role of the
    macro element: flag it iff the gradient norm of the P1 interpolant of
    the viscosity (nodal values eta_v on the finest grid) exceeds nu on at
    least one finest element it covers.  Returns (gmax, flags) keyed by
    level; gmax[L] holds the finest elements' norms."""
    nL = 2 * N
    gmax = {L: gradient_norms(Mesh(nL), eta_v)}
    flags = {}
    for l in range(L - 1, 0, -1):
        k = children_n(nL >> (L - l))
        gmax[l] = gmax[l + 1][k].max(axis=1)
        flags[l] = gmax[l] > nu
    return gmax, flags


class Hierarchy:
    def __init__(self, N: int, L: int, eta: np.ndarray, nu: float = 10.0,
                 cheb_lo: float = 0.1, cheb_hi: float = 1.1, cheb_degree: int = 2,
                 power_iters: int = 20, build_operators: bool = True, projection: str = "arithmetic",
                 eta_vertex: np.ndarray | None = None, level_coef: dict | None = None):
        nL = 2 * N
        assert nL % (1 << (L - 1)) == 0 and (nL >> (L - 1)) >= 2
        self.N, self.L, self.nu = N, L, nu
        self.cheb_lo, self.cheb_hi, self.cheb_degree = cheb_lo, cheb_hi, cheb_degree
        self.power_iters = power_iters
        self.mesh = {l: Mesh(nL >> (L - l)) for l in range(1, L + 1)}
        self.ch = {l: children(self.mesh[l], self.mesh[l + 1]) for l in range(1, L)}
        eta = np.asarray(eta, dtype=np.float64)
        assert eta.shape == (self.mesh[L].ne,)
        # viscosity hierarchy: finest values passed down (Sec. 4.2)
        self.mean, self.mx, self.mn, self.flags = {L: eta}, {L: eta}, {L: eta}, {}
        for l in range(L - 1, 0, -1):
            k = self.ch[l]
            self.mean[l] = coarse_mean(self.mean[l + 1][k], projection)
            self.mx[l] = self.mx[l + 1][k].max(axis=1)
            self.mn[l] = self.mn[l + 1][k].min(axis=1)
            self.flags[l] = self.mx[l] > nu * self.mn[l]
        if eta_vertex is not None:  # the gradient rule of Eq. 2.8 instead of the ratio rule
            self.flags = gradient_flags(N, L, eta_vertex, nu)[1]
        # DCA coefficient of coarse levels evaluated by the caller (Eq. 2.5 with
        # the analytic coefficient at the coarse element's quadrature points,
        # or the mean of its P1 interpolant, Sec. 3.2) instead of projected
        # from the children; flags keep the finest descendants' max/min
        for l, c in (level_coef or {}).items():
            assert 1 <= l < L and np.shape(c) == (self.mesh[l].ne,)
            self.mean[l] = np.asarray(c, dtype=np.float64)
        self.flist = {l: np.nonzero(self.flags[l])[0] for l in range(1, L)}
        self.findex = {}
        for l in range(1, L):
            idx = np.full(self.mesh[l].ne, -1, dtype=np.int64)
            idx[self.flist[l]] = np.arange(len(self.flist[l]))
            self.findex[l] = idx
        # stored Galerkin matrices, finest-to-coarsest (Eq. 2.7)
        self.gca = {}
        for l in range(L - 1, 0, -1):
            self.gca[l] = self._galerkin(l, self.flist[l])
        if build_operators:
            self._build_operators()

    # ---- element matrices -------------------------------------------------
    def child_matrices(self, l: int, kids: np.ndarray) -> np.ndarray:
        """Matrices C_k of level-(l+1) elements kids (any shape) as seen by
        their level-l parent."""
        shape = kids.shape
        kids = kids.ravel()
        if l + 1 == self.L:
            C = fem.element_matrices(self.mesh[self.L], self.mean[self.L][kids], kids)
        else:
            C = fem.element_matrices(self.mesh[l + 1], self.mean[l + 1][kids], kids)
            fi = self.findex[l + 1][kids]
            sel = fi >= 0
            C[sel] = self.gca[l + 1][fi[sel]]
        return C.reshape(shape + (12, 12))

    def _galerkin(self, l: int, elems: np.ndarray) -> np.ndarray:
        """A_e^GCA = sum_k (I3 x p_k)^T C_k (I3 x p_k) for elements elems."""
        if len(elems) == 0:
            return np.zeros((0, 12, 12))
        p = local_interpolation(self.mesh[l], self.mesh[l + 1], self.ch[l], elems)  # (F,8,4,4)
        P12 = np.zeros(p.shape[:2] + (12, 12))
        for c in range(3):
            P12[:, :, 4 * c:4 * c + 4, 4 * c:4 * c + 4] = p
        out = np.zeros((len(elems), 12, 12))
        chunk = 4096
        for s in range(0, len(elems), chunk):
            kids = self.ch[l][elems[s:s + chunk]]
            C = self.child_matrices(l, kids)
            Pk = P12[s:s + chunk]
            out[s:s + chunk] = np.einsum("fkia,fkij,fkjb->fab", Pk, C, Pk)
        return out

    def level_element_matrices(self, l: int) -> np.ndarray:
        """All element matrices of the level-l AGCA operator (Eq. 2.9)."""
        m = self.mesh[l]
        A = fem.element_matrices(m, self.mean[l])
        if l < self.L and len(self.flist[l]):
            A[self.flist[l]] = self.gca[l]
        return A

    # ---- level operators --------------------------------------------------
    def _build_operators(self):
        L = self.L
        self.A, self.P, self.D, self.invD, self.lam, self.mask = {}, {}, {}, {}, {}, {}
        for l in range(1, L + 1):
            m = self.mesh[l]
            self.mask[l] = fem.velocity_mask(m)
            A = fem.assemble(m, self.level_element_matrices(l))
            self.A[l] = fem.mask_matrix(A, self.mask[l], self.mask[l])
            d = self.A[l].diagonal()
            self.D[l] = d
            inv = np.zeros_like(d)
            inv[self.mask[l] > 0] = 1.0 / d[self.mask[l] > 0]
            self.invD[l] = inv
        for l in range(1, L):
            Ps = prolongation(self.mesh[l], self.mesh[l + 1])
            P = sp.block_diag([Ps, Ps, Ps]).tocsr()
            self.P[l] = fem.mask_matrix(P, self.mask[l + 1], self.mask[l])
        for l in range(2, L + 1):
            self.lam[l] = self.power_lambda(l)
        idx = np.nonzero(self.mask[1] > 0)[0]
        self.coarse_idx = idx
        Ac = self.A[1][idx][:, idx].toarray()
        self.coarse_dense = Ac
        self.coarse_factor = sla.cho_factor(Ac, lower=True)

    def power_lambda(self, l: int) -> float:
        """lambda_hat of D^-1 A_l: power iterations from the splitmix64 start
        vector, then the Rayleigh quotient (v^T A v) / (v^T D v)."""
        A, invD = self.A[l], self.invD[l]
        v = start_vector(A.shape[0]) * self.mask[l]
        for _ in range(self.power_iters):
            w = invD * (A @ v)
            v = w / np.linalg.norm(w)
        return float(v @ (A @ v)) / float(v @ (self.D[l] * v))

    def chebyshev(self, l: int, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        """Chebyshev iteration of the given degree on D^-1 A over
        [lo, hi] * lambda_hat (three-term form of the Chebyshev semi-iterative
        method)."""
        a, bb = self.cheb_lo * self.lam[l], self.cheb_hi * self.lam[l]
        theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        A, invD = self.A[l], self.invD[l]
        r = b - A @ x
        d = invD * r / theta
        x = x + d
        for _ in range(1, self.cheb_degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            r = b - A @ x
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (invD * r)
            x = x + d
            rho = rho_new
        return x

    def coarse_solve(self, b: np.ndarray) -> np.ndarray:
        x = np.zeros_like(b)
        x[self.coarse_idx] = sla.cho_solve(self.coarse_factor, b[self.coarse_idx])
        return x

    def vcycle(self, b: np.ndarray, l: int | None = None) -> np.ndarray:
        """One V-cycle for A_l x = b from x = 0 (pre- and post-smoothing with the
        same Chebyshev polynomial, so the cycle is symmetric)."""
        if l is None:
            l = self.L
        if l == 1:
            return self.coarse_solve(b)
        x = self.chebyshev(l, b, np.zeros_like(b))
        r = b - self.A[l] @ x
        bc = self.P[l - 1].T @ r
        ec = self.vcycle(bc, l - 1)
        x = x + self.P[l - 1] @ ec
        return self.chebyshev(l, b, x)

    # ---- sampled Galerkin matrices at any size ----------------------------
    def c_agca(self, l: int) -> float:
        """Fraction of flagged elements on level l (Eq. 5.7, element-wise)."""
        return float(self.flags[l].mean())


def flag_hierarchy(N: int, L: int, eta: np.ndarray, nu: float, projection: str = "arithmetic"):
    """Viscosity hierarchy and flags only (cheap at any size): dicts
    mean, mx, mn, flags keyed by level, plus the children maps."""
    nL = 2 * N
    mean, mx, mn, flags = {L: eta}, {L: eta}, {L: eta}, {}
    for l in range(L - 1, 0, -1):
        k = children_n(nL >> (L - l))
        mean[l] = coarse_mean(mean[l + 1][k], projection)
        mx[l] = mx[l + 1][k].max(axis=1)
        mn[l] = mn[l + 1][k].min(axis=1)
        flags[l] = mx[l] > nu * mn[l]
    return mean, mx, mn, flags


# Kuhn-grid vertex neighbourhood: the vertex itself and the 14 vertices it
# shares an element edge with (+-e_i, +-(e_i + e_j), +-(1, 1, 1)); the stencil
# storage of Remark 5 keeps one 3x3 block per offset
KUHN_OFFSETS = np.array([(0, 0, 0)] + [s * np.array(d) for d in
                         [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
                         for s in (1, -1)], dtype=np.int64)


def flagged_operator(H: Hierarchy, l: int):
    """The stored-Galerkin part of the level-l AGCA operator: the assembly of
    the flagged elements' matrices only (Eq. 2.9's second sum), Dirichlet
    rows and columns masked."""
    m = H.mesh[l]
    A = fem.assemble(m, H.gca[l], H.flist[l]) if len(H.flist[l]) else sp.csr_matrix((3 * m.nv, 3 * m.nv))
    return fem.mask_matrix(A, H.mask[l], H.mask[l])


def stencil_blocks(H: Hierarchy, l: int, A=None) -> np.ndarray:
    """The level-l operator (or the matrix A on the level's DoFs) as
    per-vertex stencils (Remark 5): out[v, o, c, d] is the coupling of
    component c at vertex v with component d at vertex v + KUHN_OFFSETS[o]
    (zero where the neighbour is outside the grid), read from the assembled
    global matrix."""
    m = H.mesh[l]
    n1 = m.n + 1
    A = (H.A[l] if A is None else A).tocsr()
    out = np.zeros((m.nv, len(KUHN_OFFSETS), 3, 3))
    for o, d in enumerate(KUHN_OFFSETS):
        nb = m.ijk + d
        ok = ((nb >= 0) & (nb <= m.n)).all(axis=1)
        v = np.nonzero(ok)[0]
        w = nb[ok, 0] + n1 * (nb[ok, 1] + n1 * nb[ok, 2])
        for c in range(3):
            for e in range(3):
                out[v, o, c, e] = np.asarray(A[c * m.nv + v, e * m.nv + w]).ravel()
    return out


def stencil_apply(H: Hierarchy, l: int, blocks: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A_l x from the per-vertex stencils of stencil_blocks."""
    m = H.mesh[l]
    n1 = m.n + 1
    X = x.reshape(3, m.nv).T
    Y = np.zeros((m.nv, 3))
    for o, d in enumerate(KUHN_OFFSETS):
        nb = m.ijk + d
        ok = ((nb >= 0) & (nb <= m.n)).all(axis=1)
        w = np.where(ok, nb[:, 0] + n1 * (nb[:, 1] + n1 * nb[:, 2]), 0)
        Y += np.einsum("vce,ve->vc", blocks[:, o], X[w] * ok[:, None])
    return Y.T.ravel()
