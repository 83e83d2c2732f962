"""The dense form on the tensor cores (tcgen05, split TF32) for 64-point lines,
against the FP64 oracle and against the FP32 dense form."""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev
from paper_1602_03395_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


@pytest.mark.parametrize("dims,lam,batch", [((64,), (5,), 3), ((64, 64), (7, 3), 1), ((48, 64), (4, 9), 2),
                                            ((64, 16, 64), (3, 5, 30), 1), ((64, 64, 64), (30, 30, 3), 2)])
def test_tc_field_and_density(ffx, dims, lam, batch):
    rng = np.random.default_rng(sum(dims) + batch)
    dx = (0.25,) * len(dims)
    t = 10.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    plan = ffx.Plan(dims, dx, t, lam, form="tc")
    field = ffx.ffx_expand_field(plan, to_dev(psi)).cpu().numpy()
    rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
    errs = plan.device_errors()
    forms = plan.axis_forms
    plan.close()
    ef, ed = rel_l2(field, ref), rel_l2(rho, np.abs(ref) ** 2)
    print(f"tc dims={dims} forms={forms}: field {ef:.2e} density {ed:.2e} device errors {errs}")
    assert errs == 0
    assert ef < FIELD_TOL and ed < DENSITY_TOL


def test_tc_workload_and_accumulate(ffx):
    w = inputs.config_two_cloud()
    psi = w.batch_array(3)
    ref = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, form="tc") as plan:
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, form="tc", accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
    e1, e2 = rel_l2(rho, ref), rel_l2(acc, ref.sum(0))
    print(f"tc {w.name}: density {e1:.2e}, ensemble sum {e2:.2e}")
    assert e1 < DENSITY_TOL and e2 < DENSITY_TOL


def test_tc_adjoint_and_backward(ffx):
    dims, dx, lam, t = (64, 32, 64), (0.25, 0.2, 0.3), (6, 3, 4), 3.0
    rng = np.random.default_rng(77)
    psi = random_field(rng, (2,) + dims)
    grad = rng.normal(size=(2,) + dims).astype(np.float32)
    with ffx.Plan(dims, dx, t, lam, form="tc") as plan:
        adj = ffx.ffx_expand_adjoint(plan, to_dev(psi)).cpu().numpy()
        g = ffx.ffx_expand_backward(plan, to_dev(psi), to_dev(grad)).cpu().numpy()
        assert plan.device_errors() == 0
    e1 = rel_l2(adj, O.expand_adjoint(psi, dx, t, lam))
    e2 = rel_l2(g, O.density_loss_gradient(psi, grad, dx, t, lam))
    print(f"tc adjoint {e1:.2e}, backward {e2:.2e}")
    assert e1 < FIELD_TOL and e2 < FIELD_TOL
