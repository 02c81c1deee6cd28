"""Integer-unit float helpers of the kernels (conversions between float32 and float64, and the
maximum of non-negative doubles on their bit patterns) against the C++ conversions, on the host.

tests/native/fp_bits_check.cpp includes the kernels' own header as plain C++ and checks every
float32 pattern through the widening conversion, 22 million seeded random, tie, carry and
range-edge doubles through both narrowing conversions, and 5 million maxima.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2103_11050_gb300", "csrc")


def test_fp_bits_match_cpp_conversions():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "fp_bits_check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "fp_bits_check.cpp"),
                        "-o", exe], check=True, capture_output=True, text=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok:")
