"""Helpers shared by the GPU tests: build/load the library, run it, compare."""

import numpy as np
import pytest
import torch

# relative L2 density error allowed against the FP64 oracle (FP32 path)
DENSITY_TOL = 2e-5
# the complex field carries the same FP32 rounding; its relative L2 error is
# held to the same bound
FIELD_TOL = 2e-5


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03395_gb300 import build
    build.build()
    from paper_1602_03395_gb300 import ffx
    ffx.load_library()
    return ffx


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((got - ref).ravel())
    if den == 0:
        return num
    return num / den


def to_dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_density(ffx, psi0, dims, dx, t, lam, form="auto", a=None, abar=None, accumulate=False):
    plan = ffx.Plan(dims, dx, t, lam, a, abar, form=form, accumulate=accumulate)
    try:
        out = ffx.ffx_expand(plan, to_dev(psi0))
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        plan.close()


def gpu_field(ffx, psi0, dims, dx, t, lam, form="auto", a=None, abar=None):
    plan = ffx.Plan(dims, dx, t, lam, a, abar, form=form)
    try:
        out = ffx.ffx_expand_field(plan, to_dev(psi0))
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        plan.close()


def random_field(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
