"""GB300-native AGCA multigrid (arXiv 2511.13109): adaptive Galerkin
coarse-grid approximation for the variable-viscosity Stokes problem.

The compute path is libagca (hand-written CUDA for sm_103a) behind the C ABI
of include/agca.h; this package is its thin ctypes binding plus a
torch.autograd.Function for the adjoint gradient.
"""
from .agca import (  # noqa: F401
    F32,
    F64,
    FIELD_COARSE,
    FIELD_DIAG,
    FIELD_FLAGS,
    FIELD_GCA,
    FIELD_LIST,
    FIELD_MAX,
    FIELD_MEAN,
    FIELD_MIN,
    FIELD_PMASS,
    FIELD_SIDX,
    FIELD_STENCIL,
    FP64,
    MIXED,
    PROJ_ARITHMETIC,
    PROJ_GEOMETRIC,
    PROJ_HARMONIC,
    AgcaError,
    Batch,
    Context,
    default_levels,
    exported_symbols,
    lib,
    stencil_tiles,
    stokes_apply_static,
)
from .adjoint import StokesProblem, stokes_velocity  # noqa: F401,E402
