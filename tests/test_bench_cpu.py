"""Host-side pieces of bench.py that both arms share: the level count of the
benchmark hierarchy (the reference arm computes it without loading the
library) and the config dict both arms print."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_levels_match_library(bench):
    from paper_2511_13109_gb300 import agca

    for N in (4, 8, 16, 24, 32, 48, 64, 96, 128):
        assert bench.bench_levels(N) == agca.default_levels(N), N


def test_config_of_both_arms(bench):
    cfg = bench.arm_config(64, 6, [118, 531, 2698, 14302, 11052], 1)
    assert cfg["N_pressure"] == 64 and cfg["velocity_cubes"] == 128 and cfg["levels"] == 6
    assert cfg["velocity_dofs"] == 3 * 129 ** 3 == 6440067
    assert cfg["parallelism"] == "replicas1" and cfg["global_batch"] == 1
    assert 0 < bench.FINE_STENCIL_DRAM_BYTES < 3 * 60 * 129 ** 3
