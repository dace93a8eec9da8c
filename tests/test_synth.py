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
