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


def test_binding_constants_match_the_header():
    """Every integer #define of include/bri.h that the binding mirrors has the header's value."""
    from paper_1701_00726_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "bri.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"^#define\s+BRI_([A-Z0-9_]+)\s+\(?(-?\d+)\)?", src, flags=re.M)}
    mirrored = {"OK": "BRI_OK", "NOT_CONVERGED": "BRI_NOT_CONVERGED", "PREC_F64": "PREC_F64",
                "PREC_F32": "PREC_F32", "PREC_F32_BF16": "PREC_F32_BF16", "PREC_DW": "PREC_DW",
                "ANTIPERIODIC_T": "ANTIPERIODIC_T", "KERNEL_BRILLOUIN": "KERNEL_BRILLOUIN",
                "KERNEL_WILSON": "KERNEL_WILSON", "KL_DIAGONAL": "KL_DIAGONAL", "KL_UPPER": "KL_UPPER",
                "MAX_SHIFTS": "MAX_SHIFTS"}
    for h, py in mirrored.items():
        assert defs[h] == getattr(_lib, py), h
