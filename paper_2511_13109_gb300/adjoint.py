"""Differentiable Stokes solve: velocity as a function of the element
log-viscosity theta = log(eta), with a hand-written adjoint.

Forward: set eta = exp(theta), rebuild the AGCA hierarchy (flags, Galerkin
matrices), solve K(theta) x = b.  Only the solution x is saved (the forward
solve is checkpointed; no Krylov history is stored).  Backward: K is
symmetric, so the adjoint solve K lambda = (dJ/du, 0) reuses the same
AGCA-preconditioned MINRES; the gradient is the element-wise kernel
g_e = -lambda_e^T (dA_e/dtheta_e) u_e (the element matrix of Eq. 3.5 is
linear in eta_e, so dA_e/dtheta_e = A_e).
"""
from __future__ import annotations

import torch

from .agca import FP64, Context


class StokesProblem:
    """A fixed grid, forcing and solver configuration; theta varies."""

    def __init__(self, N: int, fbar: torch.Tensor, levels: int | None = None, precision: int = FP64,
                 nu: float = 10.0, rtol: float = 1e-10, maxit: int = 20000, device="cuda",
                 rtol_adjoint: float | None = None):
        self.ctx = Context(N, levels, precision, device=device)
        self.fbar = fbar
        self.nu, self.rtol, self.maxit = nu, rtol, maxit
        # the adjoint right-hand side (dJ/du) has its own attainable residual floor
        self.rtol_adjoint = rtol if rtol_adjoint is None else rtol_adjoint
        self._theta_prepared = None  # copy of the theta the hierarchy was built for
        self.last_iters = (0, 0)

    def _prepare(self, theta: torch.Tensor):
        # the hierarchy (flags, Galerkin matrices) is rebuilt unless it was
        # built for exactly these values: an element-wise comparison on the
        # device, so two different fields can never share a hierarchy
        t = theta.detach()
        if self._theta_prepared is not None and self._theta_prepared.shape == t.shape and \
                torch.equal(self._theta_prepared, t):
            return
        self.ctx.prepare(torch.exp(t).contiguous(), self.nu)
        self._theta_prepared = t.clone()

    def solve(self, theta: torch.Tensor) -> torch.Tensor:
        self._prepare(theta)
        b = self.ctx.load_vector(self.fbar)
        x, its, _ = self.ctx.solve(b, self.rtol, self.maxit)
        self.last_iters = (its, self.last_iters[1])
        return x


class _StokesVelocity(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, problem):
        x = problem.solve(theta)
        fctx.problem = problem
        fctx.save_for_backward(theta, x)
        n3 = 3 * problem.ctx.V[problem.ctx.L]
        return x[:n3].clone()

    @staticmethod
    def backward(fctx, grad_u):
        theta, x = fctx.saved_tensors
        problem = fctx.problem
        problem._prepare(theta)
        g, its = problem.ctx.adjoint_gradient(x, grad_u.contiguous(), problem.rtol_adjoint, problem.maxit)
        problem.last_iters = (problem.last_iters[0], its)
        return g, None


def stokes_velocity(theta: torch.Tensor, problem: StokesProblem) -> torch.Tensor:
    """u(theta): finest-level velocity (SoA, 3 * V_L) of the Stokes solve."""
    return _StokesVelocity.apply(theta, problem)
