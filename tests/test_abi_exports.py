"""The C-ABI library loads and exports every function include/bri.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bri.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\**\s+\**([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bri_create", "bri_destroy", "bri_build_links", "bri_apply", "wils_apply", "kl_coeffs",
                     "sign_apply_multishift", "overlap_apply", "bri_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1701_00726_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no CUDA toolkit to build libbri.so")
        build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    # the Python binding covers the same names
    assert set(_declared()) <= set(_lib.EXPORTED)
