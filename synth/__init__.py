"""Seeded synthetic inputs for the AGCA Stokes sinker problems.

This package is shared by the CUDA path's tests/bench and by the CPU oracle.
It holds no arithmetic of the multigrid method itself: it only evaluates the
analytic viscosity and forcing fields of the sinker benchmarks (Section 3.2,
Eqs. 3.6-3.12) at element quadrature points and averages them per element.
"""
from .sinkers import (  # noqa: F401
    PERMS,
    CONFIG_SEED0,
    Problem,
    element_quadrature_points,
    cube_sinker,
    sphere_sinkers,
    sphere_sinkers_on_device,
    sphere_sinkers_vertex,
    gaussian_logbumps,
    gaussian_logbumps_on_device,
    batch_problems,
    C_UA,
    cube_field,
    sphere_field,
    field_problem,
    p1_element_means,
    level_coefficients,
    adjoint_problem,
    random_vector,
    velocity_grid,
)
