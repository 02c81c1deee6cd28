"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mpm2p.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mpm2p.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_11050_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("mpm_create", "mpm_build_basis", "mpm_eval_epsilon", "mpm_choose", "mpm_perturbation_solve",
                 "mpm_interface_solve", "mpm_downscale", "mpm_saturation_step", "mpm_step", "mpm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2103_11050_gb300 import binding
    assert sorted(binding.FUNCTIONS) == [n for n in declared()]


def test_create_rejects_bad_sizes_without_gpu_work(lib):
    from paper_2103_11050_gb300 import binding
    L = binding.load()
    h = ctypes.c_void_p()
    # non-square cells and non-positive sizes are refused before any device call
    assert L.mpm_create(ctypes.byref(h), 1, 4, 4, 1.0, 2.0, None) == binding.MPM_ERR_ARG
    assert L.mpm_create(ctypes.byref(h), 0, 4, 4, 1.0, 1.0, None) == binding.MPM_ERR_ARG
    assert L.mpm_create(ctypes.byref(h), 1, -4, 4, 1.0, 1.0, None) == binding.MPM_ERR_ARG
    assert L.mpm_create(ctypes.byref(h), 65536, 4, 4, 1.0, 1.0, None) == binding.MPM_ERR_ARG
