"""The allocation-free entry point ffx_expand_noalloc.

It serves callers that cannot call cudaMalloc while they run (a framework
that owns the device memory pool, a real-time loop); it keeps its scratch in
fixed static device arrays.  Checked through the C ABI against the regular
ffx_plan + ffx_expand path on two calls in a row (the second call reuses the
scratch the first one left behind).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

from gpu_common import DENSITY_TOL, random_field, rel_l2, require_gpu, to_dev
from paper_1602_03395_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    ("two_cloud", None),
    ("1d", None),
    ("custom", ((48, 96), (0.25, 0.2), 3.0, (7, 4), 3)),
]


def _case(name, spec):
    if name == "custom":
        dims, dx, t, lam, batch = spec
        psi = random_field(np.random.default_rng(5), (batch,) + dims)
        return dims, dx, t, lam, psi
    w = inputs.WORKLOADS[name]()
    return w.dims, w.dx, w.t, w.lam, w.batch_array(2)


@pytest.mark.parametrize("name,spec", CASES)
def test_noalloc_matches_plan_path_twice(name, spec):
    ffx = require_gpu()
    dims, dx, t, lam, psi = _case(name, spec)
    x = to_dev(psi)
    with ffx.Plan(dims, dx, t, lam) as plan:
        ref = ffx.ffx_expand(plan, x).cpu().numpy()
    lib = ffx.load_library()
    d = len(dims)
    for call in range(2):
        out = torch.full(psi.shape, float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.ffx_expand_noalloc(
            d, (ctypes.c_int64 * d)(*dims), (ctypes.c_double * d)(*dx), ctypes.c_double(t),
            (ctypes.c_int32 * d)(*lam), None, None, ctypes.c_void_p(x.data_ptr()), psi.shape[0],
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.ffx_last_error()
        got = out.cpu().numpy()
        e = rel_l2(got, ref)
        print(f"noalloc {name} call {call}: rel L2 vs ffx_expand {e:.2e}")
        assert np.isfinite(got).all()
        assert e < DENSITY_TOL


def test_noalloc_against_the_oracle():
    """The fold-form kernels the entry point always runs, against the FP64
    oracle directly (not only against the automatic-form plan path)."""
    import oracle as O
    ffx = require_gpu()
    dims, dx, t, lam = (32, 64), (0.25, 0.2), 2.5, (9, 5)
    psi = random_field(np.random.default_rng(17), (2,) + dims)
    x = to_dev(psi)
    lib = ffx.load_library()
    out = torch.full(psi.shape, float("nan"), dtype=torch.float32, device="cuda")
    rc = lib.ffx_expand_noalloc(
        2, (ctypes.c_int64 * 2)(*dims), (ctypes.c_double * 2)(*dx), ctypes.c_double(t),
        (ctypes.c_int32 * 2)(*lam), None, None, ctypes.c_void_p(x.data_ptr()), 2,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.ffx_last_error()
    e = rel_l2(out.cpu().numpy(), O.expand_density(psi, dx, t, lam))
    print(f"noalloc vs oracle: {e:.2e}")
    assert e < DENSITY_TOL


def test_noalloc_rejects_sizes_beyond_the_static_limit():
    ffx = require_gpu()
    lib = ffx.load_library()
    dims = (128, 128, 128)  # 2^21 points > FFX_NOALLOC_MAX_FIELD
    x = torch.zeros((1,) + dims, dtype=torch.complex64, device="cuda")
    out = torch.zeros((1,) + dims, dtype=torch.float32, device="cuda")
    rc = lib.ffx_expand_noalloc(3, (ctypes.c_int64 * 3)(*dims), (ctypes.c_double * 3)(0.25, 0.25, 0.25),
                                ctypes.c_double(1.0), (ctypes.c_int32 * 3)(2, 2, 2), None, None,
                                ctypes.c_void_p(x.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == ffx.FFX_EINVAL
    assert b"static field limit" in lib.ffx_last_error()
    rc = lib.ffx_expand_noalloc(1, (ctypes.c_int64 * 1)(1024), (ctypes.c_double * 1)(0.1),
                                ctypes.c_double(1.0), (ctypes.c_int32 * 1)(100), None, None,
                                ctypes.c_void_p(x.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == ffx.FFX_EINVAL
    assert b"static limit" in lib.ffx_last_error()
