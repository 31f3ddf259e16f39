"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/flare_gb.h declares (no compute calls: this runs on CPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "flare_gb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(flr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2204_12573_gb300 import build
    return build.build()


def test_header_declares_the_four_hot_path_calls():
    names = _declared()
    for f in ["flr_build_neighbors", "flr_compute_descriptors", "flr_energy_forces_uncertainty", "flr_md_step"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2204_12573_gb300 import _native as N
    assert sorted(N.EXPORTED) == sorted(n for n in _declared())


def test_version_and_error_string_without_gpu(lib_path):
    from paper_2204_12573_gb300 import _native as N
    L = N.lib()
    assert b"sm_103a" in L.flr_version()
    p = N.Params(3, 8, 3, 64, 4.5, 0.5, 0, 1)          # 3 species: rejected before any CUDA call
    h = ctypes.c_void_p()
    assert L.flr_create(ctypes.byref(p), 0, ctypes.byref(h)) == N.FLR_EINVAL
    assert b"n_species" in L.flr_last_error()
