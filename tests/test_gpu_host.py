"""ffx_expand_host: the expansion on host buffers in one C call (input copied
to the plan's staging buffer, expanded, densities copied back), against the
device-buffer call on the same plan and against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


@pytest.mark.parametrize("dims,lam,batch", [((16, 32, 48), (3, 4, 2), 3), ((64, 64, 64), (30, 30, 3), 1),
                                            ((512,), (20,), 2),
                                            ((128, 96, 128), (20, 9, 3), 2)])  # a BF16 chain
def test_host_call_equals_device_call(ffx, dims, lam, batch):
    rng = np.random.default_rng(sum(dims) + batch)
    dx, t = (0.25,) * len(dims), 6.0
    psi = random_field(rng, (batch,) + dims)
    with ffx.Plan(dims, dx, t, lam) as plan:
        dev = ffx.ffx_expand(plan, to_dev(psi)).cpu()
        h_in = torch.from_numpy(psi).pin_memory()
        h_out = torch.empty((batch,) + dims, dtype=torch.float32).pin_memory()
        ffx.ffx_expand_host(plan, h_in, h_out)
        torch.cuda.synchronize()
        assert plan.device_errors() == 0
    assert torch.equal(h_out, dev)
    e = rel_l2(h_out.numpy(), np.abs(O.expand_field(psi, dx, t, lam)) ** 2)
    print(f"host call {dims} x{batch}: density {e:.2e}")
    assert e < DENSITY_TOL


def test_host_call_accumulates_into_the_host_buffer(ffx):
    dims, dx, lam, t = (32, 48), (0.2, 0.3), (5, 3), 4.0
    rng = np.random.default_rng(9)
    psi = random_field(rng, (4,) + dims)
    ref = (np.abs(O.expand_field(psi, dx, t, lam)) ** 2).sum(axis=0)
    with ffx.Plan(dims, dx, t, lam, accumulate=True) as plan:
        out = torch.full(dims, 0.5, dtype=torch.float32)  # pageable memory works too
        ffx.ffx_expand_host(plan, torch.from_numpy(psi), out)
        torch.cuda.synchronize()
    assert rel_l2(out.numpy() - 0.5, ref) < DENSITY_TOL


def test_host_call_on_a_many_instance_plan(ffx):
    rng = np.random.default_rng(4)
    specs = [((48, 32), (0.25, 0.25), 40.0, (10, 10)), ((64,), (0.1,), 12.0, (3,)), ((96, 32, 32), (0.25,) * 3,
                                                                                  80.0, (20, 20, 20))]
    with ffx.PlanMany(specs) as plan:
        x = np.zeros(plan.points, np.complex64)
        for off, (dims, *_rest) in zip(plan.offsets, specs):
            m = int(np.prod(dims))
            x[off:off + m] = random_field(rng, (m,))
        dev = ffx.ffx_expand(plan, to_dev(x)).cpu()
        h_out = torch.empty(plan.points, dtype=torch.float32).pin_memory()
        ffx.ffx_expand_host(plan, torch.from_numpy(x).pin_memory(), h_out)
        torch.cuda.synchronize()
    assert torch.equal(h_out, dev)


def test_host_call_rejects_device_tensors(ffx):
    with ffx.Plan((64,), (0.1,), 2.0, (3,)) as plan:
        with pytest.raises(ValueError):
            ffx.ffx_expand_host(plan, torch.zeros(1, 64, dtype=torch.complex64, device="cuda"),
                                torch.empty(1, 64, dtype=torch.float32))
