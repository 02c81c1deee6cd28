"""Float64 division used on the fine-grid paths (Newton-Raphson reciprocal from a float32 seed
with a Markstein residual correction) against the IEEE division, on the GPU.

The check program (tests/native/fp64_div_check.cu) includes the library's own header, is
built with nvcc for sm_103a and compares one million seeded log-uniform quotients, the
fallback ranges of the divisor and exact cases: at most one ulp from the IEEE result.  The
same program compares the integer-unit float32/float64 conversions with the hardware ones on
a million seeded values of the float32 normal range: bit-identical.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2103_11050_gb300", "csrc")


@pytest.mark.gpu
def test_div64_within_one_ulp_of_ieee():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "fp64_div_check")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                        os.path.join(HERE, "native", "fp64_div_check.cu"), "-o", exe], check=True,
                       capture_output=True, text=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "max_ulp_div=" in out.stdout
    assert "conversion_mismatches=0" in out.stdout
