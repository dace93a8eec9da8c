"""Sinker viscosity and forcing fields, averaged per Kuhn tetrahedron.

Input format shared by every consumer:

* The unit cube is split into ``n = 2N`` cubes per axis (the velocity grid of
  the P1-iso-P2 / P1 pair, Eq. 3.3), cube ``(i, j, k)`` has lexicographic id
  ``i + n*(j + n*k)`` and is split into six tetrahedra along its main diagonal
  (Kuhn subdivision).  Tetrahedron ``t`` of a cube is
  ``{s : s[p0] >= s[p1] >= s[p2]}`` for the permutation ``PERMS[t]`` and has
  local vertices ``v0 = 0, v1 = e_p0, v2 = e_p0 + e_p1, v3 = (1, 1, 1)``.
  Element id = ``6 * cube_id + t``.
* ``eta[e]``: the element mean of the viscosity, by the symmetric 4-point
  degree-2 rule (points off the element boundary; Remark 3).  The velocity
  space is P1, so only this mean enters the bilinear form of Eq. 3.5.
* ``fbar[c, e]``: the element mean of forcing component ``c`` by the same rule.

The viscosity families follow Section 3.2 (Eqs. 3.6-3.12): ``eta_low =
DR^-0.5``, ``eta_high = DR^0.5``, forcing ``f = (0, 0, -xi)``.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
CONFIG_SEED0 = 2511131090

# symmetric 4-point rule, barycentric weights (alpha, beta, beta, beta)
_QA = 0.5854101966249685
_QB = 0.1381966011250105


@dataclasses.dataclass
class Problem:
    N: int                 # pressure cubes per axis; velocity grid has 2N
    eta: np.ndarray        # (E,) float64 element-mean viscosity
    fbar: np.ndarray       # (3, E) float64 element-mean forcing
    meta: dict


def velocity_grid(N: int) -> int:
    return 2 * N


def _ref_tets() -> np.ndarray:
    """(6, 4, 3) vertex coordinates of the six Kuhn tets of the unit cube."""
    out = np.zeros((6, 4, 3))
    for t, p in enumerate(PERMS):
        v = np.zeros(3)
        out[t, 0] = v
        for a in range(3):
            v = v.copy()
            v[p[a]] = 1.0
            out[t, a + 1] = v
    return out


def _ref_points(rule: str) -> np.ndarray:
    """(6, Q, 3) reference-cube coordinates of the evaluation points."""
    tv = _ref_tets()
    if rule == "centroid":
        return tv.mean(axis=1, keepdims=True)
    s = tv.sum(axis=1, keepdims=True)
    return _QB * s + (_QA - _QB) * tv


def element_quadrature_points(n: int, k0: int, k1: int, rule: str = "quad4",
                              device="cpu") -> torch.Tensor:
    """Points of cube layers k0..k1-1: shape (k1-k0, n, n, 6, Q, 3) in [0,1]^3.

    Axis order of the leading dims is (k, j, i) so that a C-order flatten of
    (k, j, i, t) gives the element id.
    """
    h = 1.0 / n
    ref = torch.as_tensor(_ref_points(rule), dtype=torch.float64, device=device)
    kk = torch.arange(k0, k1, dtype=torch.float64, device=device)
    jj = torch.arange(n, dtype=torch.float64, device=device)
    ii = torch.arange(n, dtype=torch.float64, device=device)
    K, J, I = torch.meshgrid(kk, jj, ii, indexing="ij")
    org = torch.stack([I, J, K], dim=-1)  # (nk, n, n, 3) as (x, y, z)
    return (org[:, :, :, None, None, :] + ref[None, None, None]) * h


def _element_means(N: int, field_fn, rule: str, device, ncomp: int):
    """Average field_fn over each element's points.  field_fn maps a (..., 3)
    point tensor to a tuple (eta, fz) of (...) tensors."""
    n = velocity_grid(N)
    E = 6 * n ** 3
    eta = np.empty(E, dtype=np.float64)
    fz = np.empty(E, dtype=np.float64)
    per_layer = 6 * n * n
    # chunk so a chunk holds at most ~8M points
    q = 1 if rule == "centroid" else 4
    nk = max(1, min(n, (8 << 20) // (per_layer * q)))
    for k0 in range(0, n, nk):
        k1 = min(n, k0 + nk)
        pts = element_quadrature_points(n, k0, k1, rule, device)
        e, f = field_fn(pts)
        eta[k0 * per_layer:k1 * per_layer] = e.mean(dim=-1).reshape(-1).cpu().numpy()
        fz[k0 * per_layer:k1 * per_layer] = f.mean(dim=-1).reshape(-1).cpu().numpy()
    fbar = np.zeros((3, E), dtype=np.float64)
    fbar[2] = fz
    return eta, fbar


def _element_means_on_device(N: int, field_fn, device):
    """As _element_means (4-point rule, one forcing component), with the
    results left on the device: (eta (E,), fbar (3, E)) float64 tensors.
    For grids whose host copies would be tens of GB."""
    n = velocity_grid(N)
    per_layer = 6 * n * n
    eta = torch.empty(6 * n ** 3, dtype=torch.float64, device=device)
    fbar = torch.zeros((3, 6 * n ** 3), dtype=torch.float64, device=device)
    nk = max(1, min(n, (8 << 20) // (per_layer * 4)))
    for k0 in range(0, n, nk):
        k1 = min(n, k0 + nk)
        e, f = field_fn(element_quadrature_points(n, k0, k1, "quad4", device))
        eta[k0 * per_layer:k1 * per_layer] = e.mean(dim=-1).reshape(-1)
        fbar[2, k0 * per_layer:k1 * per_layer] = f.mean(dim=-1).reshape(-1)
    return eta, fbar


def _device(device):
    if device == "auto":
        return "cuda" if torch.cuda.is_available() else "cpu"
    return device


def cube_sinker(N: int, lo: float = 0.375, hi: float = 0.625, eta_in: float = 1e3,
                eta_out: float = 1.0, device="cpu") -> Problem:
    """One cube sinker [lo, hi]^3 (eta_1 of Eq. 3.6 with explicit levels),
    evaluated at element centroids; f = (0, 0, -1) inside."""

    def fn(x):
        inside = ((x >= lo) & (x <= hi)).all(dim=-1)
        eta = torch.where(inside, torch.full_like(x[..., 0], eta_in), torch.full_like(x[..., 0], eta_out))
        return eta, -inside.to(torch.float64)

    eta, fbar = _element_means(N, fn, "centroid", _device(device), 1)
    return Problem(N, eta, fbar, dict(kind="cube", lo=lo, hi=hi, eta_in=eta_in, eta_out=eta_out))


def _tanh_spheres_fn(centres: np.ndarray, radii: np.ndarray, width: float, dr: float):
    eta_hi, eta_lo = dr ** 0.5, dr ** -0.5

    def fn(x):
        c = torch.as_tensor(centres, dtype=torch.float64, device=x.device)
        xi = torch.zeros_like(x[..., 0])
        for j in range(c.shape[0]):
            d = torch.linalg.vector_norm(x - c[j], dim=-1)
            xi = torch.maximum(xi, 0.5 * (1.0 - torch.tanh((d - float(radii[j])) / width)))
        return eta_lo + (eta_hi - eta_lo) * xi, -xi

    return fn


def sphere_sinkers(N: int, n_sinkers: int = 8, radius: float = 0.08, width: float = 0.01,
                   dr: float = 1e6, seed: int = CONFIG_SEED0 + 1, device="cpu") -> Problem:
    """Union of tanh-smoothed balls (the eta_4 / eta_6 shapes of Eq. 3.6 with a
    tanh transition of the given width), centres uniform in [0.2, 0.8]^3."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(n_sinkers, 3))
    radii = np.full(n_sinkers, radius)
    fn = _tanh_spheres_fn(centres, radii, width, dr)
    eta, fbar = _element_means(N, fn, "quad4", _device(device), 1)
    return Problem(N, eta, fbar, dict(kind="spheres", centres=centres, radius=radius,
                                      width=width, dr=dr, seed=seed))


def sphere_sinkers_on_device(N: int, n_sinkers: int = 8, radius: float = 0.08, width: float = 0.01,
                             dr: float = 1e6, seed: int = CONFIG_SEED0 + 1, device="cuda"):
    """The sphere_sinkers field family generated and kept on the device:
    (eta, fbar, centres) with eta (E,) and fbar (3, E) float64 tensors."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(n_sinkers, 3))
    fn = _tanh_spheres_fn(centres, np.full(n_sinkers, radius), width, dr)
    eta, fbar = _element_means_on_device(N, fn, device)
    return eta, fbar, centres


def sphere_sinkers_vertex(N: int, n_sinkers: int = 8, radius: float = 0.08, width: float = 0.01,
                          dr: float = 1e6, seed: int = CONFIG_SEED0 + 1) -> np.ndarray:
    """The sphere_sinkers viscosity at the vertices of the finest grid (the
    nodal values of its P1 interpolant), float64 in vertex order
    i + (n+1)(j + (n+1)k)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(n_sinkers, 3))
    fn = _tanh_spheres_fn(centres, np.full(n_sinkers, radius), width, dr)
    n = velocity_grid(N)
    g = torch.arange(n + 1, dtype=torch.float64) / n
    K, J, I = torch.meshgrid(g, g, g, indexing="ij")
    eta, _ = fn(torch.stack([I, J, K], dim=-1))
    return eta.reshape(-1).numpy()


def _logbump_params(n_bumps: int, seed: int):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_bumps, 3))
    amps = rng.uniform(-3.0, 3.0, size=n_bumps)
    widths = rng.uniform(0.03, 0.15, size=n_bumps)
    return centres, amps, widths


def _logbump_fn(centres: np.ndarray, amps: np.ndarray, widths: np.ndarray):
    def fn(x):
        c = torch.as_tensor(centres, dtype=torch.float64, device=x.device)
        lg = torch.zeros_like(x[..., 0])
        for k in range(len(amps)):
            r2 = ((x - c[k]) ** 2).sum(dim=-1)
            lg = lg + float(amps[k]) * torch.exp(-r2 / (2.0 * float(widths[k]) ** 2))
        lg = lg.clamp(-3.0, 3.0)
        return torch.pow(10.0, lg), -(lg + 3.0) / 6.0

    return fn


def gaussian_logbumps(N: int, n_bumps: int = 20, seed: int = CONFIG_SEED0 + 2,
                      device="cpu") -> Problem:
    """Smooth log10-viscosity: sum of Gaussian bumps (centres uniform in
    [0, 1]^3, amplitudes uniform in [-3, 3], widths uniform in [0.03, 0.15]),
    clipped to [-3, 3]; forcing f_z = -(log10 mu + 3) / 6 (a constant forcing
    would be a pure gradient and give u = 0)."""
    centres, amps, widths = _logbump_params(n_bumps, seed)
    eta, fbar = _element_means(N, _logbump_fn(centres, amps, widths), "quad4", _device(device), 1)
    return Problem(N, eta, fbar, dict(kind="logbumps", centres=centres, amps=amps,
                                      widths=widths, seed=seed))


def gaussian_logbumps_on_device(N: int, n_bumps: int = 20, seed: int = CONFIG_SEED0 + 2, device="cuda"):
    """The gaussian_logbumps field generated and kept on the device: (eta (E,),
    fbar (3, E)) float64 tensors (the host copies at N = 128 would be 3 GB)."""
    centres, amps, widths = _logbump_params(n_bumps, seed)
    return _element_means_on_device(N, _logbump_fn(centres, amps, widths), device)


# centre of the grid-unaligned shapes of Section 3.2
C_UA = 11.0 / 24.0


def cube_field(kind: str, dr: float, omega: float = 10.0):
    """The cube viscosities of Eqs. 3.6-3.9 as a field function x -> (eta,
    f_z): "aligned" (eta_1, the cube of half-width 1/8 around 1/2), "unaligned"
    (eta_2, around C_UA = 11/24) or "tanh" (eta_3, the product of the 1-D tanh
    profiles of Eq. 3.7 around C_UA with smoothing omega); eta = eta_low +
    (eta_high - eta_low) xi with eta_high/low = DR^(+-1/2), f = (0, 0, -xi)."""
    eta_hi, eta_lo = dr ** 0.5, dr ** -0.5
    r = 0.125

    def fn(x):
        if kind == "tanh":
            xi = torch.ones_like(x[..., 0])
            for a in range(3):
                xi = xi * 0.5 * (torch.tanh(omega * (x[..., a] - (C_UA - r))) - torch.tanh(omega * (x[..., a] - (C_UA + r))))
        else:
            c = 0.5 if kind == "aligned" else C_UA
            xi = ((x - c).abs() <= r).all(dim=-1).to(torch.float64)
        return eta_lo + (eta_hi - eta_lo) * xi, -xi

    return fn


def sphere_field(centres: np.ndarray, radii: np.ndarray, width: float, dr: float):
    """Union of tanh-smoothed balls as a field function x -> (eta, f_z)."""
    return _tanh_spheres_fn(np.asarray(centres, dtype=np.float64), np.asarray(radii, dtype=np.float64), width, dr)


def field_problem(N: int, fn, kind: str = "field", device="cpu") -> Problem:
    """Element means (4-point rule) of a field function on the finest grid."""
    eta, fbar = _element_means(N, fn, "quad4", _device(device), 1)
    return Problem(N, eta, fbar, dict(kind=kind))


def p1_element_means(n: int, fn) -> np.ndarray:
    """Mean over each Kuhn tetrahedron of a grid with n cubes per axis of the
    P1 interpolant of the field (its values at the grid vertices): the mean
    of a linear function is the average of its 4 vertex values."""
    g = torch.arange(n + 1, dtype=torch.float64) / n
    K, J, I = torch.meshgrid(g, g, g, indexing="ij")
    vals, _ = fn(torch.stack([I, J, K], dim=-1))
    vals = vals.numpy()                                  # [k][j][i]
    out = np.zeros((n, n, n, 6))
    for t, p in enumerate(PERMS):
        corner = np.zeros(3, dtype=np.int64)
        acc = vals[:n, :n, :n].copy()
        for a in range(3):
            corner[p[a]] += 1
            acc = acc + vals[corner[2]:corner[2] + n, corner[1]:corner[1] + n, corner[0]:corner[0] + n]
        out[..., t] = acc * 0.25
    return out.reshape(-1)


def level_coefficients(fn, N: int, L: int, mode: str = "analytic") -> dict:
    """Coefficients of the coarse levels l = 1..L-1 (level l has 2N / 2^(L-l)
    cubes per axis) evaluated on the level's own elements, for direct coarse
    approximation (Eq. 2.5): "analytic" = the field's mean over the 4-point
    rule of the coarse element, "p1" = the mean of its P1 interpolant on the
    coarse grid (Sec. 3.2)."""
    out = {}
    for l in range(1, L):
        n = (2 * N) >> (L - l)
        if mode == "analytic":
            assert n % 2 == 0
            out[l], _ = _element_means(n // 2, fn, "quad4", "cpu", 1)
        elif mode == "p1":
            out[l] = p1_element_means(n, fn)
        else:
            raise ValueError(mode)
    return out


def batch_problems(seed: int = CONFIG_SEED0 + 3, sizes=(32, 48, 64), per_size: int = 8,
                   device="cpu", generate=True):
    """Independent single-sphere problems of uneven sizes: centre uniform in
    [0.2, 0.8]^3, radius uniform in [0.05, 0.15], DR = 10^k with k uniform in
    {2..6}, tanh width 0.01.  Returns a list of Problem (or of parameter dicts
    when generate=False)."""
    rng = np.random.default_rng(seed)
    Ns = np.repeat(np.asarray(sizes), per_size)
    rng.shuffle(Ns)
    out = []
    for N in Ns:
        centre = rng.uniform(0.2, 0.8, size=(1, 3))
        r = rng.uniform(0.05, 0.15)
        k = int(rng.integers(2, 7))
        params = dict(N=int(N), centre=centre, radius=float(r), dr=10.0 ** k, width=0.01)
        if not generate:
            out.append(params)
            continue
        fn = _tanh_spheres_fn(centre, np.array([r]), 0.01, 10.0 ** k)
        eta, fbar = _element_means(int(N), fn, "quad4", _device(device), 1)
        out.append(Problem(int(N), eta, fbar, dict(kind="sphere", **params)))
    return out


def adjoint_problem(N: int, seed: int = CONFIG_SEED0 + 4, device="cpu"):
    """The 8-sphere setup with jump 1e4 and a perturbed log-viscosity field used
    to produce the observation: returns (problem, theta_obs) where theta_obs =
    log(eta) + N(0, 0.1^2) per element."""
    p = sphere_sinkers(N, dr=1e4, seed=CONFIG_SEED0 + 1, device=device)
    rng = np.random.default_rng(seed)
    theta_obs = np.log(p.eta) + rng.normal(0.0, 0.1, size=p.eta.shape)
    return p, theta_obs


def random_vector(size: int, seed: int) -> np.ndarray:
    """Uniform [-1, 1] float64 test vector."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=size)
