"""FP64 / FP32 arithmetic throughput of the device (tests/probes/alu_probe.cu).

The FP64 stencil is bounded by min(HBM, FP64 ALU); this probe measures the
FP64 FMA rate that bound uses and checks the FP64 : FP32 ratio the design
relies on (FP64 far below FP32 on this GPU generation)."""
import os
import re
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_alu_probe(capsys):
    src = os.path.join(HERE, "probes", "alu_probe.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_probe")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    with capsys.disabled():
        print("\n" + out)
    fp64 = float(re.search(r"fp64 fma_tinstr_s ([0-9.]+)", out).group(1))
    fp32 = float(re.search(r"fp32 fma_tinstr_s ([0-9.]+)", out).group(1))
    assert fp64 > 0 and fp32 > 0
    assert fp64 < fp32 / 8, (fp64, fp32)
