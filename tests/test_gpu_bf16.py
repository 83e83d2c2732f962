"""BF16 operands on the tensor cores (FFX_TC_BF16, kind::f16), against the
FP64 oracle.

Split: every operand value v becomes hi = bf16(v), lo = bf16(v - hi), and the
products X_hi T_hi + X_hi T_lo + X_lo T_hi are accumulated in FP32.  The
representation error of hi + lo is at most 2^-18 |v| and the dropped lo*lo
term at most 2^-18 of each product, so the field's relative error per pass is
a few 2^-18 (~1e-5 worst case, ~1e-6 for rounding errors of random sign),
within the FP32 path's 2e-5 density bar, which these tests hold it to.

Unsplit (with FFX_TC_UNSPLIT): one product on operands rounded to BF16
(u = 2^-9 each): ~2^-9 relative per pass of random-sign rounding, about
sqrt(d) that over d passes and twice that on the density: ~5e-3 for d = 3.
That is the reported BF16 class; the tests hold it to 1e-2 and print it.

Each case also checks that the BF16 kernel really ran: its result is not the
split-TF32 one bit for bit."""

import numpy as np
import pytest

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

BF16_UNSPLIT_TOL = 1e-2

CASES = [
    ((128, 96, 256), (9, 5, 3), 1),   # whole row blocks (128, 256), a half block (96); strided and contiguous
    ((64, 64, 64), (30, 30, 3), 24),  # 64-point passes with more than four items per block
    ((16, 1024), (4, 7), 2),          # 1024-point lines (the 16-point axis: FP32)
    ((256, 32), (100, 6), 3),         # lam = 100 on a strided 256-point axis; 32-point lines keep TF32
    ((128, 48), (7, 5), 2),           # a stride of 48 lines: per-thread loads instead of bulk copies
]


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


def density(ffx, dims, dx, t, lam, psi, **kw):
    with ffx.Plan(dims, dx, t, lam, form="tc", **kw) as plan:
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    return rho


@pytest.mark.parametrize("dims,lam,batch", CASES)
def test_split_bf16_density(ffx, dims, lam, batch):
    rng = np.random.default_rng(sum(dims) + batch)
    dx, t = (0.25,) * len(dims), 10.0
    psi = random_field(rng, (batch,) + dims)
    ref = np.abs(O.expand_field(psi, dx, t, lam)) ** 2
    rho_b = density(ffx, dims, dx, t, lam, psi, bf16=True)
    rho_t = density(ffx, dims, dx, t, lam, psi)
    eb, et = rel_l2(rho_b, ref), rel_l2(rho_t, ref)
    print(f"split bf16 {dims} x{batch}: density {eb:.2e} (split tf32 {et:.2e})")
    assert eb < DENSITY_TOL
    assert not np.array_equal(rho_b, rho_t)


def test_split_bf16_workload_geometry(ffx):
    """The large two-cloud geometry (lam = 100, t = 400, dx = 0.25) on a 128^3
    lattice, with the two-cloud input: the magnitudes the headline passes see."""
    from paper_1602_03395_gb300 import inputs
    dims, dx, lam, t = (128, 128, 128), (0.25,) * 3, (100, 100, 100), 400.0
    psi = inputs.two_cloud_3d(np.random.default_rng(3), dims).astype(np.complex64)[None]
    ref = np.abs(O.expand_field(psi, dx, t, lam)) ** 2
    rho = density(ffx, dims, dx, t, lam, psi, bf16=True)
    e = rel_l2(rho, ref)
    print(f"split bf16 two-cloud 128^3 lam 100: density {e:.2e}")
    assert e < DENSITY_TOL


def test_split_bf16_field_accumulate_backward_adjoint(ffx):
    dims, dx, lam, t = (96, 64, 128), (0.25, 0.2, 0.3), (6, 3, 4), 3.0
    rng = np.random.default_rng(77)
    psi = random_field(rng, (3,) + dims)
    grad = rng.normal(size=(3,) + dims).astype(np.float32)
    g_in = random_field(rng, (3,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True) as plan:
        x = to_dev(psi)
        f = ffx.ffx_expand_field(plan, x).cpu().numpy()
        g = ffx.ffx_expand_backward(plan, x, to_dev(grad)).cpu().numpy()
        adj = ffx.ffx_expand_adjoint(plan, to_dev(g_in)).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    e_f = rel_l2(f, ref)
    e_acc = rel_l2(acc, (np.abs(ref) ** 2).sum(0))
    e_g = rel_l2(g, O.density_loss_gradient(psi, grad, dx, t, lam))
    e_a = rel_l2(adj, O.expand_adjoint(g_in, dx, t, lam))
    print(f"split bf16 {dims}: field {e_f:.2e}, ensemble sum {e_acc:.2e}, backward {e_g:.2e}, adjoint {e_a:.2e}")
    assert e_f < FIELD_TOL and e_acc < DENSITY_TOL and e_g < FIELD_TOL and e_a < FIELD_TOL


@pytest.mark.parametrize("dims,lam,batch", CASES[:2])
def test_unsplit_bf16_reported_class(ffx, dims, lam, batch):
    rng = np.random.default_rng(5 + batch)
    dx, t = (0.25,) * len(dims), 10.0
    psi = random_field(rng, (batch,) + dims)
    ref = np.abs(O.expand_field(psi, dx, t, lam)) ** 2
    rho_b = density(ffx, dims, dx, t, lam, psi, bf16=True, unsplit=True)
    rho_t = density(ffx, dims, dx, t, lam, psi, unsplit=True)
    eb, et = rel_l2(rho_b, ref), rel_l2(rho_t, ref)
    print(f"unsplit bf16 {dims} x{batch}: density {eb:.2e} (unsplit tf32 {et:.2e})")
    assert eb < BF16_UNSPLIT_TOL
    assert eb > et  # BF16 rounding, not TF32


def test_bf16_flag_checks(ffx):
    with pytest.raises(ffx.FfxError) as ei:
        ffx.Plan((64, 64), (0.25, 0.25), 1.0, (3, 3), form="fold", bf16=True)
    assert ei.value.code == ffx.FFX_EINVAL


# BF16 chains: lattices whose lines per realization are not multiples of the
# 128-line tile (tiles straddle realizations), 2-D and 3-D, density, field and
# ensemble sum
CHAIN_CASES = [
    ((96, 192), (5, 9), 3),
    ((128, 96, 192), (30, 4, 7), 2),
]


@pytest.mark.parametrize("dims,lam,batch", CHAIN_CASES)
def test_bf16_chain_density_field_accumulate(ffx, dims, lam, batch):
    rng = np.random.default_rng(11 * batch + len(dims))
    dx, t = (0.25,) * len(dims), 10.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True) as plan:
        assert plan.bf16_chain(batch)
        assert plan.pass_order() == tuple(reversed(range(len(dims))))
        x = to_dev(psi)
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        f = ffx.ffx_expand_field(plan, x).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, accumulate=True) as plan:
        assert plan.bf16_chain(batch)
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, unsplit=True) as plan:
        assert plan.bf16_chain(batch)
        rho_u = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    dens = np.abs(ref) ** 2
    e_d, e_f = rel_l2(rho, dens), rel_l2(f, ref)
    e_acc, e_u = rel_l2(acc, dens.sum(0)), rel_l2(rho_u, dens)
    print(f"bf16 chain {dims} x{batch}: density {e_d:.2e}, field {e_f:.2e}, ensemble sum {e_acc:.2e}, "
          f"unsplit density {e_u:.2e}")
    assert e_d < DENSITY_TOL and e_f < FIELD_TOL and e_acc < DENSITY_TOL and e_u < BF16_UNSPLIT_TOL
    # the density is |field|^2 of the same chain (to FP32 rounding)
    assert rel_l2(rho, np.abs(f) ** 2) < 1e-6


def test_bf16_pass_splits_contiguous_fp32_input(ffx):
    """Per-axis path (the 32-point axes keep TF32, so no chain): the BF16 pass
    along the last axis first splits its contiguous FP32 lines into BF16
    planes (one more launch), for densities, fields, the ensemble sum and the
    adjoint half of the backward pass."""
    dims, lam, batch = (32, 32, 256), (5, 6, 20), 3
    rng = np.random.default_rng(2024)
    dx, t = (0.25, 0.25, 0.3), 10.0
    psi = random_field(rng, (batch,) + dims)
    grad = rng.normal(size=(batch,) + dims).astype(np.float32)
    ref = O.expand_field(psi, dx, t, lam)
    dens = np.abs(ref) ** 2
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True) as plan:
        assert not plan.bf16_chain(batch)
        x = to_dev(psi)
        n0 = plan.launch_count()
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        assert plan.launch_count() - n0 == len(dims) + 1  # the passes and the split
        f = ffx.ffx_expand_field(plan, x).cpu().numpy()
        g = ffx.ffx_expand_backward(plan, x, to_dev(grad)).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    e_d, e_f, e_acc = rel_l2(rho, dens), rel_l2(f, ref), rel_l2(acc, dens.sum(0))
    e_g = rel_l2(g, O.density_loss_gradient(psi, grad, dx, t, lam))
    print(f"bf16 split first pass {dims} x{batch}: density {e_d:.2e}, field {e_f:.2e}, ensemble sum {e_acc:.2e}, "
          f"backward {e_g:.2e}")
    assert e_d < DENSITY_TOL and e_f < FIELD_TOL and e_acc < DENSITY_TOL and e_g < FIELD_TOL


@pytest.mark.parametrize("dims,lam,batch", CHAIN_CASES)
def test_bf16_chain_backward(ffx, dims, lam, batch):
    """Backward calls on BF16-chain plans: the forward field (a chain except on
    2-D plans), then the adjoint half as a chain -- the split of 2 g psi into
    BF16 planes and the T_j^H passes from the last axis to the first -- per
    realization and with the batch's shared gradient of an ensemble-sum plan,
    against the oracle's gradient; the launches the call makes."""
    rng = np.random.default_rng(5 * batch + len(dims))
    dx, t = (0.25,) * len(dims), 10.0
    d = len(dims)
    psi = random_field(rng, (batch,) + dims)
    grad = rng.normal(size=(batch,) + dims).astype(np.float32)
    gsum = rng.normal(size=dims).astype(np.float32)
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True) as plan:
        assert plan.bf16_chain(batch)
        x = to_dev(psi)
        n0 = plan.launch_count()
        g = ffx.ffx_expand_backward(plan, x, to_dev(grad)).cpu().numpy()
        # forward: the chain's split and d passes, or on 2-D plans the per-axis
        # passes with the split of the contiguous axis's FP32 lines; adjoint:
        # the gradient split and d passes
        assert plan.launch_count() - n0 == 2 * d + 2
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, accumulate=True) as plan:
        assert plan.bf16_chain(batch)
        gs = ffx.ffx_expand_backward(plan, to_dev(psi), to_dev(gsum)).cpu().numpy()
        assert plan.device_errors() == 0
    e_g = rel_l2(g, O.density_loss_gradient(psi, grad, dx, t, lam))
    ref_s = np.stack([O.density_loss_gradient(psi[b:b + 1], gsum[None], dx, t, lam)[0] for b in range(batch)])
    e_s = rel_l2(gs, ref_s)
    print(f"bf16 chain backward {dims} x{batch}: {e_g:.2e}, shared gradient {e_s:.2e}")
    assert e_g < FIELD_TOL and e_s < FIELD_TOL
