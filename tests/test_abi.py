"""The C ABI library builds, loads and exports every entry point that
include/agca.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "agca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(agca_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libagca():
    from paper_2511_13109_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    assert "agca_create" in names and "agca_solve" in names and len(names) >= 20


def test_library_exports_every_declared_symbol(libagca):
    for name in _declared():
        assert hasattr(libagca, name), name


def test_binding_covers_header():
    from paper_2511_13109_gb300 import agca

    assert sorted(agca.exported_symbols()) == _declared()


def test_host_only_calls(libagca):
    """Creation, sizing and argument validation run on the host only."""
    from paper_2511_13109_gb300 import agca

    L = agca.lib()
    h = ctypes.c_void_p()
    assert L.agca_create(16, 4, 0, None, ctypes.byref(h)) == 0
    sz = ctypes.c_size_t()
    assert L.agca_workspace_size(h, ctypes.byref(sz)) == 0 and sz.value > 0
    # misaligned or short workspaces are rejected before any device access
    assert L.agca_bind_workspace(h, ctypes.c_void_p(8), sz.value) == 1
    assert L.agca_bind_workspace(h, ctypes.c_void_p(256), 16) == 2
    # calls out of order report a state error
    assert L.agca_setup(h) == 7
    assert L.agca_set_level_coefficient(h, 1, ctypes.c_void_p(256)) == 7   # before agca_flag
    assert L.agca_set_level_coefficient(h, 4, ctypes.c_void_p(256)) == 1   # the finest level is not coarse
    assert L.agca_set_smoother(h, 1, 0.3, 1.2, 20) == 1
    assert b"smoother" in L.agca_last_error(h)
    assert L.agca_set_solver_options(h, 0.0, 4) == 1
    assert L.agca_set_solver_options(h, 1e-4, 0) == 1
    assert L.agca_set_solver_options(h, 1e-4, 8) == 0
    assert L.agca_flag_gradient(h, None, ctypes.c_double(1.0), ctypes.byref(sz)) == 1  # nodal viscosity missing
    assert L.agca_set_coarse_projection(h, 3) == 1 and L.agca_set_coarse_projection(h, -1) == 1
    assert L.agca_set_coarse_projection(h, 2) == 0 and L.agca_set_coarse_projection(h, 0) == 0
    assert L.agca_set_tile_config(h, 2, 1, 8, 5) == 0
    assert L.agca_set_tile_config(h, 2, 1, 12, 0) == 1   # 12 block rows: FP32 cycle launches only
    assert L.agca_set_tile_config(h, 0, 1, 8, 0) == 1
    assert L.agca_set_tile_config(h, 2, 6, 8, 0) == 1
    by, zc = ctypes.c_int(), ctypes.c_int()
    assert L.agca_tile_config(h, 2, 1, ctypes.byref(by), ctypes.byref(zc)) == 0 and (by.value, zc.value) == (8, 5)
    L.agca_destroy(h)
    bad = ctypes.c_void_p()
    assert L.agca_create(16, 6, 0, None, ctypes.byref(bad)) == 1   # 32 cubes cannot coarsen 5 times to >= 2
    assert L.agca_create(5, 3, 0, None, ctypes.byref(bad)) == 1    # 10 cubes cannot be halved twice
    assert L.agca_create(4, 2, 7, None, ctypes.byref(bad)) == 1    # unknown precision
    assert L.agca_create(512, 3, 0, None, ctypes.byref(bad)) == 1  # beyond 32-bit kernel indexing


def test_default_levels():
    from paper_2511_13109_gb300 import agca

    assert [agca.default_levels(N) for N in (16, 32, 48, 64, 128)] == [4, 5, 5, 6, 7]
