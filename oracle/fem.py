"""Finite-element pieces of the Stokes demonstrator (Section 3.1).

Velocity: P1 on the level-L Kuhn mesh, three components; pressure: P1 on the
level-(L-1) mesh (the P1-iso-P2 / P1 pair, Eq. 3.3).  Vectors are SoA: the
velocity DoF (component c, vertex v) has index c*V + v.  Local element DoF
(vertex a, component c) has index c*4 + a.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh


def element_matrices(mesh: Mesh, coef: np.ndarray, elems=None) -> np.ndarray:
    """Local viscous matrices of Eq. 3.5 for element-constant viscosity:
    [A_e]_{(a,c),(b,d)} = coef_e |T| (delta_cd g_a.g_b + g_{a,d} g_{b,c}),
    i.e. the integral of 2 eta eps(phi_a e_c) : eps(phi_b e_d).
    Returns (E', 12, 12) in local index c*4 + a."""
    if elems is None:
        elems = np.arange(mesh.ne)
    G = mesh.grads[elems]                                # (E',4,3)
    vol = mesh.volumes[elems]
    gg = np.einsum("eai,ebi->eab", G, G)                 # g_a . g_b
    A = np.zeros((len(elems), 3, 4, 3, 4))
    for c in range(3):
        A[:, c, :, c, :] += gg
    A += np.einsum("ead,ebc->ecadb", G, G)               # g_{a,d} g_{b,c}
    A *= (np.asarray(coef)[..., None, None, None, None] * vol[:, None, None, None, None])
    return A.reshape(len(elems), 12, 12)


def element_dofs(mesh: Mesh, elems=None) -> np.ndarray:
    """(E', 12) global DoF index of each local DoF c*4 + a."""
    if elems is None:
        elems = np.arange(mesh.ne)
    v = mesh.tets[elems]                                 # (E',4)
    return np.concatenate([v + c * mesh.nv for c in range(3)], axis=1)


def assemble(mesh: Mesh, mats: np.ndarray, elems=None) -> sp.csr_matrix:
    """Sum_e I_e A_e I_e^T (Eq. 2.3) as an explicit sparse matrix."""
    dofs = element_dofs(mesh, elems)
    rows = np.repeat(dofs, 12, axis=1).ravel()
    cols = np.tile(dofs, (1, 12)).ravel()
    n = 3 * mesh.nv
    return sp.coo_matrix((mats.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def velocity_mask(mesh: Mesh) -> np.ndarray:
    """1.0 on interior velocity DoFs, 0.0 on Dirichlet ones (g = 0)."""
    return np.tile(mesh.interior.astype(np.float64), 3)


def mask_matrix(A: sp.spmatrix, mrow: np.ndarray, mcol: np.ndarray) -> sp.csr_matrix:
    return (sp.diags(mrow) @ A @ sp.diags(mcol)).tocsr()


def load_vector(mesh: Mesh, fbar: np.ndarray, elems=None) -> np.ndarray:
    """b_{(a,c)} = sum_T |T| fbar_c(T) / 4 for element-constant forcing, masked.
    elems: sum over these elements only (fbar[:, i] belongs to elems[i])."""
    if elems is None:
        elems = np.arange(mesh.ne)
    b = np.zeros(3 * mesh.nv)
    w = mesh.volumes[elems] / 4.0
    for c in range(3):
        np.add.at(b, c * mesh.nv + mesh.tets[elems].ravel(), np.repeat(w * fbar[c], 4))
    return b * velocity_mask(mesh)


def load_vector_quadrature(mesh: Mesh, f) -> np.ndarray:
    """b_{(a,c)} = sum_T sum_q w_q f_c(x_q) phi_a(x_q) with the 4-point rule."""
    alpha, beta = 0.5854101966249685, 0.1381966011250105
    X = mesh.coords[mesh.tets]                           # (E,4,3)
    S = X.sum(axis=1, keepdims=True)
    Q = beta * S + (alpha - beta) * X                    # (E,4,3) point q near vertex q
    F = f(Q.reshape(-1, 3)).reshape(mesh.ne, 4, 3)       # f at points
    phi = np.full((4, 4), beta)
    np.fill_diagonal(phi, alpha)                         # phi_a(x_q)
    w = mesh.volumes / 4.0
    b = np.zeros(3 * mesh.nv)
    for c in range(3):
        contrib = np.einsum("qa,eq->ea", phi, F[:, :, c]) * w[:, None]
        np.add.at(b, c * mesh.nv + mesh.tets.ravel(), contrib.ravel())
    return b * velocity_mask(mesh)


def divergence(pmesh: Mesh, vmesh: Mesh, parent: np.ndarray, elems=None) -> sp.csr_matrix:
    """D_kj = int psi_k div Phi_j (Eq. 3.5, second line), exact by the centroid
    rule on the velocity tets (psi_k is linear there, div Phi_j constant).
    Shape (V_p, 3 V_v); velocity columns are not masked.  elems: sum over
    these velocity elements only (parent is indexed by velocity element)."""
    if elems is None:
        elems = np.arange(vmesh.ne)
    G = vmesh.grads[elems]                               # (E,4,3)
    lam = pmesh.barycentric(parent[elems], vmesh.centroids[elems])  # (E,4) psi at centroid
    pv = pmesh.tets[parent[elems]]                       # (E,4) pressure vertices
    vol = vmesh.volumes[elems]
    tv = vmesh.tets[elems]
    rows, cols, vals = [], [], []
    for m in range(4):
        for c in range(3):
            for a in range(4):
                rows.append(pv[:, m])
                cols.append(c * vmesh.nv + tv[:, a])
                vals.append(vol * lam[:, m] * G[:, a, c])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.coo_matrix((vals, (rows, cols)), shape=(pmesh.nv, 3 * vmesh.nv)).tocsr()


def pressure_mass_lumped(pmesh: Mesh, eta_fine: np.ndarray, ch: np.ndarray, elems=None) -> np.ndarray:
    """Viscosity-weighted lumped pressure mass: M_ii = sum_{T ni i} w_T |T| / 4,
    w_T = mean of 1/eta over the 8 velocity elements refining T.  elems: sum
    over these pressure elements only (row i of ch are the children of
    elems[i], as indices into eta_fine)."""
    if elems is None:
        elems = np.arange(pmesh.ne)
    inv = 1.0 / eta_fine[ch]                             # (E_p, 8)
    w = ((inv[:, 0] + inv[:, 1]) + (inv[:, 2] + inv[:, 3])) + ((inv[:, 4] + inv[:, 5]) + (inv[:, 6] + inv[:, 7]))
    w = w * 0.125
    M = np.zeros(pmesh.nv)
    np.add.at(M, pmesh.tets[elems].ravel(), np.repeat(w * pmesh.volumes[elems] / 4.0, 4))
    return M
