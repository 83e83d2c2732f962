"""The C-ABI library builds, loads and exports every symbol include/ffx.h
declares; host-side argument checks answer without touching a GPU."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "ffx.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ffx_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1602_03395_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["ffx_plan", "ffx_expand", "ffx_expand_field", "ffx_expand_backward",
                 "ffx_expand_adjoint", "ffx_plan_destroy", "ffx_error_string", "ffx_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_host_argument_checks(lib):
    """These calls fail in host-side validation, before any CUDA call."""
    lib.ffx_plan.restype = ctypes.c_int
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 1)(64)
    dx = (ctypes.c_double * 1)(0.2)
    lam = (ctypes.c_int32 * 1)(3)
    assert lib.ffx_plan(ctypes.byref(h), 0, dims, dx, ctypes.c_double(1.0), lam, None, None, 0) == 1
    bad = (ctypes.c_int32 * 1)(0)
    assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(1.0), bad, None, None, 0) == 1
    odd = (ctypes.c_int64 * 1)(100)
    assert lib.ffx_plan(ctypes.byref(h), 1, odd, dx, ctypes.c_double(1.0), lam, None, None, 0) == 4
    assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(float("nan")), lam, None, None, 0) == 1
    assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(1.0), lam, None, None, 0x400) == 1
    assert h.value is None
    lib.ffx_last_error.restype = ctypes.c_char_p
    assert b"flag" in lib.ffx_last_error()
    # operand flags: BF16 with a non-tensor-core form, BF16 and TF32 together
    assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(1.0), lam, None, None, 0x100 | 0x2) == 1
    assert b"FFX_TC_BF16" in lib.ffx_last_error()
    assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(1.0), lam, None, None, 0x100 | 0x200) == 1
    assert b"exclude" in lib.ffx_last_error()
    # the unsplit tensor-core variant exists for the tensor-core form only
    for form in (0x0, 0x2, 0x3):
        assert lib.ffx_plan(ctypes.byref(h), 1, dims, dx, ctypes.c_double(1.0), lam, None, None, 0x80 | form) == 1
        assert b"FFX_FORM_TC" in lib.ffx_last_error()
    assert h.value is None
    lib.ffx_error_string.restype = ctypes.c_char_p
    assert lib.ffx_error_string(1) == b"invalid argument"
    lib.ffx_supported_length.argtypes = [ctypes.c_int64]
    assert lib.ffx_supported_length(512) == 1 and lib.ffx_supported_length(100) == 0
    # null plan is rejected by every call taking one
    lib.ffx_expand.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p]
    assert lib.ffx_expand(None, None, 1, None, None) == 1
    assert lib.ffx_plan_destroy(None) == 0


def test_many_plan_flag_checks(lib):
    """Many-instance plans reject the flags that do not apply to them, and the
    operand flags outside the tensor-core forms, before any CUDA call."""
    from paper_1602_03395_gb300.ffx import InstanceDesc
    descs = (InstanceDesc * 1)()
    descs[0].ndim = 1
    descs[0].dims[0] = 64
    descs[0].spacing[0] = 0.2
    descs[0].magnification[0] = 3
    descs[0].t = 1.0
    lib.ffx_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    for flags, text in [(0x10, b"ACCUMULATE"), (0x20, b"flag"), (0x40, b"flag"), (0x80 | 0x4, b"flag"),
                        (0x100 | 0x200, b"exclude"), (0x200 | 0x2, b"FFX_FORM_TC"), (0x100 | 0x3, b"FFX_FORM_TC")]:
        assert lib.ffx_plan_many(ctypes.byref(h), 1, descs, ctypes.c_uint32(flags)) == 1, hex(flags)
        assert text in lib.ffx_last_error(), (hex(flags), lib.ffx_last_error())
        assert h.value is None
