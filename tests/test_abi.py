"""The C ABI: the library builds for sm_103a, loads, and exports every entry
point that include/vtm.h declares.  No compute call (no GPU needed)."""
import ctypes
import os
import re

import pytest


@pytest.fixture(scope="module")
def lib(root_dir):
    from paper_0910_0663_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared(root_dir):
    text = open(os.path.join(root_dir, "include", "vtm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vtm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary(root_dir):
    names = _declared(root_dir)
    for must in ("vtm_plan", "vtm_factor", "vtm_solve", "vtm_adjoint", "vtm_set_values",
                 "vtm_destroy", "vtm_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib, root_dir):
    for name in _declared(root_dir):
        assert hasattr(lib, name), name


def test_binding_exposes_the_same_names(lib, root_dir):
    from paper_0910_0663_gb300 import _vtm
    for name in _declared(root_dir):
        assert hasattr(_vtm, name), name


def test_strerror_without_gpu(lib):
    lib.vtm_strerror.restype = ctypes.c_char_p
    assert lib.vtm_strerror(0) == b"success"
    assert b"converge" in lib.vtm_strerror(-4) or b"limit" in lib.vtm_strerror(-4)


def test_null_arguments_are_rejected_without_gpu(lib):
    lib.vtm_plan.restype = ctypes.c_int
    out = ctypes.c_void_p()
    # n <= 0 and NULL arrays are refused before any CUDA call
    assert lib.vtm_plan(ctypes.c_int64(0), None, None, None, None, 1, ctypes.c_double(1.0), None,
                        None, ctypes.byref(out)) == -1
    lib.vtm_factor.restype = ctypes.c_int
    assert lib.vtm_factor(None) == -1
