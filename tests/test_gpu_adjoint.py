"""Adjoint gradient of J = 0.5 ||u - u_obs||^2 with respect to the element
log-viscosity, through torch.autograd: against the oracle's direct adjoint
and against central finite differences of the forward solve."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from oracle import stokes as ostokes
from synth import sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


def _setup(N, prec, dr=1e4):
    p = sphere_sinkers(N, 2, 0.2, 0.05, dr)
    fbar = torch.from_numpy(p.fbar.ravel()).to(DEV)
    prob = pkg.StokesProblem(N, fbar, precision=prec, rtol=1e-12, device=DEV)
    theta = torch.log(torch.from_numpy(p.eta).to(DEV))
    return p, prob, theta


@pytest.mark.parametrize("N", [4, 8])
@pytest.mark.parametrize("prec", [pkg.FP64, pkg.MIXED])
def test_adjoint_matches_oracle(prec, N):
    p, prob, theta = _setup(N, prec)
    rng = np.random.default_rng(11)
    L = prob.ctx.L
    H = oagca.Hierarchy(N, L, p.eta, 10.0)
    S = ostokes.Stokes(H)
    u_obs = rng.normal(size=S.nu_) * S.mask * 1e-3
    th = theta.clone().requires_grad_(True)
    u = pkg.stokes_velocity(th, prob)
    J = 0.5 * torch.sum((u - torch.from_numpy(u_obs).to(DEV)) ** 2)
    J.backward()
    g = th.grad.cpu().numpy()
    x = S.direct(S.rhs(p.fbar))
    g_ref = S.adjoint_gradient(x, u_obs)
    assert np.abs(g - g_ref).max() <= 1e-8 * np.abs(g_ref).max()


def test_adjoint_matches_oracle_16():
    """16^3 pressure cubes (32^3 velocity cubes, 4 levels), mixed precision.
    The oracle's sparse LU does not finish in minutes at this size, so its
    forward and adjoint solves run its own MINRES to a 1e-12 relative
    residual, as the GPU solves do (asserted to 1e-10 of max |g|)."""
    N = 16
    p, prob, theta = _setup(N, pkg.MIXED)
    H = oagca.Hierarchy(N, prob.ctx.L, p.eta, 10.0)
    S = ostokes.Stokes(H)
    u_obs = np.random.default_rng(13).normal(size=S.nu_) * S.mask * 1e-3
    th = theta.clone().requires_grad_(True)
    u = pkg.stokes_velocity(th, prob)
    (0.5 * torch.sum((u - torch.from_numpy(u_obs).to(DEV)) ** 2)).backward()
    g = th.grad.cpu().numpy()
    x, _ = S.solve(S.rhs(p.fbar), 1e-12)
    g_ref = S.adjoint_gradient(x, u_obs, solver="minres", rtol=1e-12)
    # measured on a GB300: 1.1e-13 of max |g|
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max()


def _fd4(J, theta, d, eps):
    """Fourth-order central difference of J along d (truncation O(eps^4), so
    directions whose derivative nearly cancels are still resolved)."""
    return (8.0 * (J(theta + eps * d) - J(theta - eps * d)) - (J(theta + 2 * eps * d) - J(theta - 2 * eps * d))) / \
        (12.0 * eps)


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.MIXED])
def test_adjoint_matches_finite_differences(prec):
    N = 8
    p, prob, theta = _setup(N, prec)
    rng = np.random.default_rng(12)
    n3 = 3 * prob.ctx.V[prob.ctx.L]
    with torch.no_grad():
        u0 = pkg.stokes_velocity(theta, prob)
    # observation from a perturbed log-viscosity (sigma 0.1 per element)
    th_obs = theta + 0.1 * torch.from_numpy(rng.normal(size=theta.numel())).to(DEV)
    with torch.no_grad():
        u_obs = pkg.stokes_velocity(th_obs, prob).clone()

    def J(th):
        with torch.no_grad():
            u = pkg.stokes_velocity(th, prob)
            return 0.5 * float(torch.sum((u - u_obs) ** 2))

    th = theta.clone().requires_grad_(True)
    u = pkg.stokes_velocity(th, prob)
    Jt = 0.5 * torch.sum((u - u_obs) ** 2)
    Jt.backward()
    g = th.grad.clone()
    eps = 1e-4
    for k in range(32):  # 32 seeded directions
        d = torch.from_numpy(np.random.default_rng(100 + k).normal(size=theta.numel())).to(DEV)
        fd = _fd4(J, theta, d, eps)
        ad = float(torch.dot(g, d))
        assert abs(fd - ad) <= 1e-5 * abs(fd), (k, fd, ad)
    assert u0.shape == (n3,)


# directions per precision at 64^3 (four forward solves each): 16 for the
# mixed solver, 2 for the FP64 one (its 1e-10 solves take ~6x longer); the
# 32 directions of the adjoint configuration run at 8^3 above
FULL_DIRECTIONS = {"mixed": 16, "fp64": 2}


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_adjoint_full_size_finite_differences(prec):
    """The adjoint benchmark workload (64^3 pressure cubes, 8 spheres, jump
    1e4, observation from log-viscosity + N(0, 0.1^2)): the autograd gradient
    against central finite differences of the forward solve along seeded
    directions.  Forward solves go to a 1e-10 relative residual (the FP64
    floor of this field at 64^3 is 4.4e-11), the adjoint solve to 1e-9 (its
    right-hand side u - u_obs has its own floor).  The fourth-order central
    difference then resolves a directional derivative to about 1e-9
    absolute: its noise (the solves' errors divided by eps, 1.3e-9 measured
    at eps = 1e-3) and its truncation (eps^4, 4.8e-9 measured at eps = 1e-2)
    balance near eps = 4e-3.  Each direction must agree to 1e-5 of the
    larger of its own derivative and the root mean square over the
    directions, so a direction whose derivative nearly cancels (|dJ| ~ 1e-5
    against a typical 1e-3) is held to the finite difference's resolution;
    the count of directions within 1e-5 of their own derivative is printed."""
    from synth import adjoint_problem

    N = 64
    p, theta_obs = adjoint_problem(N)
    fbar = torch.from_numpy(p.fbar.ravel()).to(DEV)
    precision = pkg.MIXED if prec == "mixed" else pkg.FP64
    prob = pkg.StokesProblem(N, fbar, precision=precision, rtol=1e-10, maxit=60000, device=DEV, rtol_adjoint=1e-9)
    theta = torch.log(torch.from_numpy(p.eta).to(DEV))
    with torch.no_grad():
        u_obs = pkg.stokes_velocity(torch.from_numpy(theta_obs).to(DEV), prob).clone()

    def J(th):
        with torch.no_grad():
            u = pkg.stokes_velocity(th, prob)
            return 0.5 * float(torch.sum((u - u_obs) ** 2))

    th = theta.clone().requires_grad_(True)
    u = pkg.stokes_velocity(th, prob)
    (0.5 * torch.sum((u - u_obs) ** 2)).backward()
    g = th.grad.clone()
    assert torch.isfinite(g).all()
    eps = 4e-3
    pairs = []
    for k in range(FULL_DIRECTIONS[prec]):
        d = torch.from_numpy(np.random.default_rng(200 + k).normal(size=theta.numel())).to(DEV)
        pairs.append((_fd4(J, theta, d, eps), float(torch.dot(g, d))))
    fds = np.array([f for f, _ in pairs])
    rms = float(np.sqrt(np.mean(fds ** 2)))
    strict = sum(abs(f - a) <= 1e-5 * abs(f) for f, a in pairs)
    worst = max(abs(f - a) / max(abs(f), rms) for f, a in pairs)
    print(f"\n64^3 adjoint ({prec}): {len(pairs)} directions, rms derivative {rms:.3e}, worst difference "
          f"{worst:.2e} of max(|dJ|, rms); {strict} of {len(pairs)} within 1e-5 of their own derivative")
    for k, (f, a) in enumerate(pairs):
        assert abs(f - a) <= 1e-5 * max(abs(f), rms), (k, f, a, rms)
