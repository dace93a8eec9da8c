"""The paper's own outer solver (Sec. 4) for the Stokes system of Eq. 3.4:
FGMRES, right-preconditioned by the upper block-triangular preconditioner of
Eq. 4.1 with the diag(A)-BFBT Schur-complement approximation of Eq. 4.2.

Test infrastructure only (imported by tests, never by the library).

Sign reading: with K = [[A, B^T], [B, 0]] (B = -D as in oracle.stokes) the
Schur complement is -S, S = B A^-1 B^T, and the block-triangular
preconditioner is Q = [[A~, B^T], [0, -S~]], so that with exact blocks
K Q^-1 = [[I, 0], [B A^-1, I]] and FGMRES ends in two steps.  The printed
Eq. 4.1 carries the signs of the paper's own convention for B.

The pressure is determined up to a constant; Z = B W^-1 B^T is singular on
the constants, so its solves run on the mean-zero subspace (first pressure
DoF pinned, result projected), and solutions are compared after removing
the pressure mean.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .stokes import Stokes


class BlockTriangular:
    """Q^-1 of Eq. 4.1 with S~^-1 the diag(A)-BFBT of Eq. 4.2:
    S~^-1 = Z^-1 (B W^-1 A W^-1 B^T) Z^-1,  W = diag(A),  Z = B W^-1 B^T.
    a_inv: the velocity-block approximate inverse (default one AGCA V-cycle);
    s_inv: override of S~^-1 (default BFBT); A_bfbt: override of the A inside
    the BFBT middle factor (default the Stokes velocity block)."""

    def __init__(self, S: Stokes, a_inv=None, s_inv=None, A_bfbt=None):
        self.S = S
        d = S.A.diagonal()
        self.winv = np.where(S.mask > 0, 1.0 / np.where(d != 0.0, d, 1.0), 0.0)
        self.A_bfbt = S.A if A_bfbt is None else A_bfbt
        self.Z = (S.B @ sp.diags(self.winv) @ S.BT).tocsc()
        self._zlu = spla.splu(self.Z[1:, 1:].tocsc())
        self.a_inv = a_inv if a_inv is not None else S.h.vcycle
        self.s_inv = s_inv if s_inv is not None else self.bfbt

    def z_solve(self, r):
        """Z^-1 on the mean-zero subspace (the range of the symmetric Z)."""
        r = r - r.mean()
        x = np.zeros_like(r)
        x[1:] = self._zlu.solve(r[1:])
        return x - x.mean()

    def bfbt(self, rp):
        t = self.z_solve(rp)
        t = self.S.B @ (self.winv * (self.A_bfbt @ (self.winv * (self.S.BT @ t))))
        return self.z_solve(t)

    def __call__(self, r):
        ru, rp = self.S.split(r)
        zp = -self.s_inv(rp)
        zu = self.a_inv(ru - self.S.BT @ zp)
        return np.concatenate([zu, zp])


def fgmres(K, b, precond, rtol=1e-8, restart=50, maxit=2000):
    """Flexible GMRES (Saad 1993): right preconditioning by a map that may
    change between iterations, Arnoldi with modified Gram-Schmidt, the small
    least-squares problem solved afresh each step.  Stops when the residual
    norm |b - K x| has dropped to rtol |b|.  Returns (x, iterations)."""
    n = len(b)
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    its = 0
    if nb == 0.0:
        return x, 0
    while its < maxit:
        r = b - K(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            break
        V = [r / beta]
        Zs = []
        H = np.zeros((restart + 1, restart))
        y = np.zeros(0)
        for j in range(restart):
            z = precond(V[j])
            Zs.append(z)
            w = K(z)
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0.0 else w)
            g = np.zeros(j + 2)
            g[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], g, rcond=None)[0]
            res = np.linalg.norm(g - H[:j + 2, :j + 1] @ y)
            its += 1
            if res <= rtol * nb or H[j + 1, j] == 0.0 or its >= maxit:
                break
        x = x + sum(yi * zi for yi, zi in zip(y, Zs))
    return x, its


def solve(S: Stokes, b, rtol=1e-8, restart=50, maxit=2000, precond=None):
    """FGMRES with Q^-1 (V-cycle and BFBT by default); pressure mean removed."""
    Q = precond if precond is not None else BlockTriangular(S)
    x, its = fgmres(S.K, b, Q, rtol, restart, maxit)
    x[S.nu_:] = S.project(x[S.nu_:])
    return x, its
