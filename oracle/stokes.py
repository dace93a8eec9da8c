"""Stokes saddle-point system (Eq. 3.4), MINRES with a block-diagonal
preconditioner (Remark 6), a sparse direct reference solve and the adjoint
gradient with respect to the element log-viscosity.

Unknowns x = [u; p]: u on the level-L velocity mesh (SoA, Dirichlet DoFs
zero), p on the level-(L-1) pressure mesh (all vertices).  B = -D with
D_kj = int psi_k div Phi_j, so that K = [[A, B^T], [B, 0]] is symmetric and p
has the physical sign of Eq. 3.2.  The pressure is fixed up to a constant:
results are compared after removing the plain mean over pressure DoFs.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .agca import Hierarchy


class Stokes:
    def __init__(self, hier: Hierarchy):
        self.h = hier
        L = hier.L
        vm, pm = hier.mesh[L], hier.mesh[L - 1]
        self.vm, self.pm = vm, pm
        ch = hier.ch[L - 1]
        parent = np.empty(vm.ne, dtype=np.int64)
        parent[ch.ravel()] = np.repeat(np.arange(pm.ne), 8)
        self.parent = parent
        self.mask = hier.mask[L]
        D = fem.divergence(pm, vm, parent)
        self.B = -(D @ sp.diags(self.mask)).tocsr()
        self.BT = self.B.T.tocsr()
        self.A = hier.A[L]
        self.Mp = fem.pressure_mass_lumped(pm, hier.mean[L], ch)
        self.nu_ = 3 * vm.nv
        self.np_ = pm.nv

    # ---- operators ---------------------------------------------------------
    def split(self, x):
        return x[:self.nu_], x[self.nu_:]

    def K(self, x):
        u, p = self.split(x)
        return np.concatenate([self.A @ u + self.BT @ p, self.B @ u])

    @staticmethod
    def project(p):
        return p - p.mean()

    def precondition(self, r):
        """blockdiag(V-cycle on A, Pi M_{1/eta}^-1 Pi) with Pi the mean-zero
        projection of the pressure."""
        ru, rp = self.split(r)
        zu = self.h.vcycle(ru)
        zp = self.project(self.project(rp) / self.Mp)
        return np.concatenate([zu, zp])

    def rhs(self, fbar):
        b = np.zeros(self.nu_ + self.np_)
        b[:self.nu_] = fem.load_vector(self.vm, fbar)
        return b

    # ---- solvers -----------------------------------------------------------
    def minres(self, b, rtol, maxit, x0=None):
        """Preconditioned MINRES on K with this preconditioner (see minres)."""
        return minres(self.K, self.precondition, b, rtol, maxit, x0=x0)

    def solve(self, b, rtol=1e-8, inner_rtol=1e-10, maxit=2000, max_outer=20):
        """Residual refinement around MINRES until the true residual satisfies
        ||b - K x||_2 <= rtol ||b||_2 (Eq. 4.3 with the requested tolerance)."""
        x = np.zeros_like(b)
        nb = np.linalg.norm(b)
        its = 0
        for _ in range(max_outer):
            r = b - self.K(x)
            if np.linalg.norm(r) <= rtol * nb:
                break
            d, k = self.minres(r, inner_rtol, maxit)
            its += k
            x = x + d
            x[self.nu_:] = self.project(x[self.nu_:])
        return x, its

    def direct(self, b):
        """Sparse LU of K on interior velocity DoFs and all pressure DoFs but
        the first (pinned), then the mean-zero pressure."""
        iv = np.nonzero(self.mask > 0)[0]
        Aii = self.A[iv][:, iv]
        Bi = self.B[1:][:, iv]
        Kr = sp.bmat([[Aii, Bi.T], [Bi, None]]).tocsc()
        rhs = np.concatenate([b[iv], b[self.nu_ + 1:]])
        sol = spla.splu(Kr).solve(rhs)
        x = np.zeros_like(b)
        x[iv] = sol[:len(iv)]
        x[self.nu_ + 1:] = sol[len(iv):]
        x[self.nu_:] = self.project(x[self.nu_:])
        return x

    # ---- adjoint -----------------------------------------------------------
    def element_sensitivity(self, lam_u, u):
        """s_e = lambda_e^T (dA/dtheta_e) u_e with theta = log(eta): the element
        matrix of Eq. 3.5 is linear in eta_e, so dA_e/dtheta_e = A_e."""
        eta = self.h.mean[self.h.L]
        Ke = fem.element_matrices(self.vm, eta)          # (E,12,12)
        dofs = fem.element_dofs(self.vm)
        return np.einsum("ei,eij,ej->e", lam_u[dofs], Ke, u[dofs])

    def adjoint_gradient(self, x, u_obs, solver="direct", rtol=1e-13):
        """dJ/dtheta for J = 0.5 ||u - u_obs||^2: solve K lambda = (u - u_obs, 0)
        (K symmetric), then g_e = -lambda_e^T (dA_e/dtheta_e) u_e.  solver:
        "direct" (sparse LU) or MINRES to the relative residual rtol."""
        u = x[:self.nu_]
        rhs = np.zeros_like(x)
        rhs[:self.nu_] = (u - u_obs) * self.mask
        lam = self.direct(rhs) if solver == "direct" else self.solve(rhs, rtol)[0]
        return -self.element_sensitivity(lam[:self.nu_], u)


def minres(K, precondition, b, rtol, maxit, x0=None, dot=np.dot):
    """Preconditioned MINRES (Lanczos in the preconditioner inner product,
    Givens QR of the tridiagonal; Remark 6's symmetric alternative to FGMRES).
    Stops when the preconditioned residual norm |eta| has dropped by rtol.
    dot(a, b) is the Euclidean inner product (a sum over all ranks when the
    vectors are distributed).  Returns (x, iterations)."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    v_old = np.zeros(n)
    v = b - K(x)
    z = precondition(v)
    gamma = np.sqrt(max(dot(v, z), 0.0))
    gamma_old = 1.0
    eta = gamma
    eta0 = gamma
    s_old = s = 0.0
    c_old = c = 1.0
    w_old = np.zeros(n)
    w = np.zeros(n)
    it = 0
    if gamma == 0.0:
        return x, 0
    while it < maxit and abs(eta) > rtol * eta0:
        it += 1
        z = z / gamma
        Kz = K(z)
        delta = dot(Kz, z)
        v_new = Kz - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = precondition(v_new)
        gamma_new = np.sqrt(max(dot(v_new, z_new), 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = np.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        v_old, v, z = v, v_new, z_new
        gamma_old, gamma = gamma, gamma_new
        w_old, w = w, w_new
        c_old, c, s_old, s = c, c_new, s, s_new
        if gamma == 0.0:
            break
    return x, it
