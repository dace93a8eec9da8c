"""The device-resident generator gives the same inputs as the host one."""
import numpy as np
import torch

from synth import sphere_sinkers, sphere_sinkers_on_device


def test_on_device_generator_matches_host_generator():
    p = sphere_sinkers(6, 3, 0.15, 0.02, 1e5, seed=9)
    eta, fbar, centres = sphere_sinkers_on_device(6, 3, 0.15, 0.02, 1e5, seed=9, device="cpu")
    assert isinstance(eta, torch.Tensor) and eta.dtype == torch.float64
    assert np.array_equal(eta.numpy(), p.eta)
    assert np.array_equal(fbar.numpy(), p.fbar)
    assert np.array_equal(centres, p.meta["centres"])


def test_vertex_values_are_the_field_at_the_vertices():
    """Nodal values in vertex order: the corner vertex (0,0,0) and a vertex
    at a sinker centre (rounded to the grid) against the field formula."""
    from synth import sphere_sinkers_vertex

    v = sphere_sinkers_vertex(4, 2, 0.2, 0.05, 1e4, seed=3)
    assert v.shape == (9 ** 3,) and v.dtype == np.float64
    assert np.isclose(v.min(), 1e-2, rtol=1e-6) and v.max() <= 1e2 * (1 + 1e-12)
    # monotone in the distance to the nearest centre: the largest value sits at the vertex closest to a centre
    centres = np.random.default_rng(3).uniform(0.2, 0.8, size=(2, 3))
    g = np.arange(9) / 8.0
    K, J, I = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    d = np.min(np.linalg.norm(pts[:, None, :] - centres[None], axis=2), axis=1)
    assert np.argmax(v) == np.argmin(d)


def test_on_device_logbumps_match_host_generator():
    from synth import gaussian_logbumps, gaussian_logbumps_on_device

    p = gaussian_logbumps(5, n_bumps=6, seed=4)
    eta, fbar = gaussian_logbumps_on_device(5, n_bumps=6, seed=4, device="cpu")
    assert np.array_equal(eta.numpy(), p.eta)
    assert np.array_equal(fbar.numpy(), p.fbar)
    assert p.eta.min() >= 1e-3 * (1 - 1e-12) and p.eta.max() <= 1e3 * (1 + 1e-12)
