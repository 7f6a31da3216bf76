"""The exact per-row rounding of the CUDA library, checked on the host: the
64.64 reciprocal floor(z * 2^64 / f) and the ceiling ceil(v * z / f) it
drives (the prediction of Eq. 4 per row) against 128-bit integer division,
on edge and 2 million random operands.  nvcc compiles the helpers as host
code; no GPU is needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_exact_rounding_helpers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "rounding_check"
    src = os.path.join(HERE, "native", "rounding_check.cu")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", src, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
