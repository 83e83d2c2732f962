"""The one-launch forward map of small lattices (every axis <= 64 points,
dense form): against the FP64 oracle, and bit for bit against the per-axis
launches it replaces."""

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


CASES = [((64, 64, 64), (30, 30, 3), 1), ((64, 64, 64), (30, 30, 3), 2), ((64, 64, 64), (30, 30, 3), 3), ((32, 48), (7, 5), 2),
         ((16, 64, 32), (3, 40, 9), 1), ((48, 16), (11, 2), 700), ((64, 32, 16), (5, 6, 7), 37)]


@pytest.mark.parametrize("dims,lam,batch", CASES)
def test_fused_matches_oracle_and_unfused(ffx, dims, lam, batch):
    rng = np.random.default_rng(sum(dims) * 7 + batch)
    dx, t = (0.25,) * len(dims), 12.0
    psi = random_field(rng, (batch,) + dims)
    with ffx.Plan(dims, dx, t, lam, form="dense") as fused, \
            ffx.Plan(dims, dx, t, lam, form="dense", fused=False) as plain:
        assert fused.fused and not plain.fused
        assert fused.launches_per_call() == 1 and plain.launches_per_call() == len(dims)
        # batches past the fused limit take the per-axis launches (same results)
        assert fused.launches_per_call(batch=batch) == (1 if batch <= fused.fused_max_batch else len(dims))
        if dims == (64, 64, 64):
            assert fused.fused_max_batch == 2
        x = to_dev(psi)
        rho_f = ffx.ffx_expand(fused, x).cpu().numpy()
        rho_p = ffx.ffx_expand(plain, x).cpu().numpy()
        fld_f = ffx.ffx_expand_field(fused, x).cpu().numpy()
        fld_p = ffx.ffx_expand_field(plain, x).cpu().numpy()
        assert fused.device_errors() == 0
    # small batches against the oracle; every batch against the unfused launches
    if batch <= 40:
        ref = O.expand_field(psi, dx, t, lam)
        ef, ed = rel_l2(fld_f, ref), rel_l2(rho_f, np.abs(ref) ** 2)
        print(f"fused {dims} x{batch}: field {ef:.2e} density {ed:.2e}")
        assert ef < FIELD_TOL and ed < DENSITY_TOL
    assert np.array_equal(rho_f, rho_p)
    assert np.array_equal(fld_f, fld_p)


def test_fused_workload_accumulate_and_in_place(ffx):
    w = inputs.config_two_cloud()
    psi = w.batch_array(5)
    ref = O.expand_field(psi, w.dx, w.t, w.lam)
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, accumulate=True) as plan:
        assert plan.fused
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        acc2 = ffx.ffx_expand(plan, to_dev(psi), torch.from_numpy(acc).cuda()).cpu().numpy()
    with ffx.Plan(w.dims, w.dx, w.t, w.lam) as plan:
        assert plan.fused
        x = to_dev(psi)
        ffx.ffx_expand_field(plan, x, x)  # in place
        fld = x.cpu().numpy()
        assert plan.device_errors() == 0
    e1 = rel_l2(acc, (np.abs(ref) ** 2).sum(0))
    e2 = rel_l2(acc2, 2 * (np.abs(ref) ** 2).sum(0))
    e3 = rel_l2(fld, ref)
    print(f"fused {w.name}: ensemble {e1:.2e}, ensemble added twice {e2:.2e}, in-place field {e3:.2e}")
    assert e1 < DENSITY_TOL and e2 < DENSITY_TOL and e3 < FIELD_TOL


def test_fusion_applies_only_to_short_dense_axes(ffx):
    with ffx.Plan((64,), (0.25,), 5.0, (9,), form="dense") as p1:
        assert not p1.fused
    with ffx.Plan((64, 128), (0.25, 0.25), 5.0, (9, 3), form="dense") as p2:
        assert not p2.fused
    with ffx.Plan((64, 64), (0.25, 0.25), 5.0, (9, 3), form="fold") as p3:
        assert not p3.fused
    with ffx.Plan((64, 64), (0.25, 0.25), 5.0, (9, 3), form="dense", fused=False) as p4:
        assert not p4.fused


@pytest.mark.parametrize("dims,lam,batch", [((64, 64, 64), (30, 30, 3), 1), ((64, 64), (7, 5), 3),
                                            ((64, 64), (7, 5), 8)])
def test_fused_tensor_core_launch(ffx, dims, lam, batch):
    """Axes of 64 points under the automatic form: the fused launch on the
    tensor cores (split TF32), against the oracle; fields, densities, the
    ensemble sum and an in-place field."""
    rng = np.random.default_rng(sum(dims) + 3 * batch)
    dx, t = (0.25,) * len(dims), 9.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam) as plan:
        assert plan.fused and batch <= plan.fused_max_batch
        assert plan.call_forms(batch) == ("tc",) * len(dims)
        x = to_dev(psi)
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        fld = ffx.ffx_expand_field(plan, x).cpu().numpy()
        y = x.clone()
        ffx.ffx_expand_field(plan, y, y)
        inplace = y.cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
    ef, ed = rel_l2(fld, ref), rel_l2(rho, np.abs(ref) ** 2)
    ea, ei = rel_l2(acc, (np.abs(ref) ** 2).sum(0)), rel_l2(inplace, ref)
    print(f"fused tc {dims} x{batch}: field {ef:.2e} density {ed:.2e} ensemble {ea:.2e} in place {ei:.2e}")
    assert max(ef, ei) < FIELD_TOL and max(ed, ea) < DENSITY_TOL
