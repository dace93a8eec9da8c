"""Source-level invariants of the CUDA library, checked on the host."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2511_13109_gb300", "csrc")


def test_every_kernel_waits_for_its_predecessor():
    """Kernels are launched with programmatic stream serialization, so a
    kernel may start before the one ahead of it in the stream has finished;
    each must therefore begin with grid_dep_entry() (griddepcontrol.wait)
    before it touches memory the earlier kernel writes."""
    missing, seen = [], 0
    for path in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        src = open(path).read()
        for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?(\w+)\s*\(", src):
            body = src[src.index("{", m.end()) + 1:]
            first = body.lstrip().split(";", 1)[0]
            seen += 1
            if "grid_dep_entry()" not in first:
                missing.append(f"{os.path.basename(path)}:{m.group(1)}")
    assert seen > 30
    assert not missing, missing
