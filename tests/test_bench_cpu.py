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
    cfg = bench.arm_config("logbump", 128, 7, [0, 1, 2, 3, 4, 5], 1)
    assert cfg["N_pressure"] == 128 and cfg["velocity_cubes"] == 256 and cfg["levels"] == 7
    assert cfg["velocity_dofs"] == 3 * 257 ** 3 == 50923779
    assert cfg["pressure_dofs"] == 129 ** 3 == 2146689
    assert cfg["parallelism"] == "replicas1" and cfg["global_batch"] == 1
    assert "128^3 pressure cubes" in cfg["workload"]


def test_fp64_peak_from_unit_counts(bench):
    # 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz, the nominal 1.25 TFLOP/s
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-4


def test_reference_arm_names_the_size_it_times(bench, capsys):
    class A:
        steps, warmup, gpus, field, N = 1, 0, 1, "logbump", 128

    assert bench.run_reference(A()) == 0
    import json

    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["N_pressure"] == 16
    assert line["config"]["velocity_dofs"] == 3 * 33 ** 3
    assert "128^3" in line["config"]["sample_of"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
