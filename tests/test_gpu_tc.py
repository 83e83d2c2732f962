"""The dense form on the tensor cores (tcgen05, split TF32) for axes whose
length is a multiple of 16 from 32 up (a last row block narrower than 128 real
rows when 2N is not a multiple of 128), against the FP64 oracle."""

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


TC_CASES = [
    ((64,), (5,), 3),
    ((64, 64), (7, 3), 1),
    ((48, 64), (4, 9), 2),
    ((64, 16, 64), (3, 5, 30), 1),
    ((64, 64, 64), (30, 30, 3), 2),
    # longer axes: several row blocks per line, ragged line tiles, strided axes
    ((128,), (3,), 300),
    ((192, 48), (5, 2), 3),
    ((256, 96), (4, 7), 1),
    ((48, 384), (3, 6), 2),
    ((512, 32), (3, 4), 1),
    ((768,), (5,), 2),
    ((1024,), (3,), 5),
    ((128, 16, 192), (9, 4, 3), 1),
    # lengths whose last row block is partial (2N mod 128 = 32, 64, 96)
    ((96, 96, 96), (10, 10, 10), 1),
    ((48, 48, 48), (20, 20, 20), 2),
    ((32,), (50,), 200),
    ((128, 32, 32), (15, 15, 15), 1),
    ((384, 96), (3, 7), 2),
]


@pytest.mark.parametrize("dims,lam,batch", TC_CASES)
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


@pytest.mark.parametrize("dims", [(64, 32, 64), (96, 48, 32)])
def test_tc_adjoint_and_backward(ffx, dims):
    dx, lam, t = (0.25, 0.2, 0.3), (6, 3, 4), 3.0
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


@pytest.mark.parametrize("dims,lam", [((128, 64), (5, 3)), ((256,), (7,)), ((16, 192), (3, 4))])
def test_tc_accumulate_and_backward_long_axes(ffx, dims, lam):
    rng = np.random.default_rng(sum(dims))
    dx, t, batch = (0.25,) * len(dims), 6.0, 3
    psi = random_field(rng, (batch,) + dims)
    grad = rng.normal(size=(batch,) + dims).astype(np.float32)
    ref = np.abs(O.expand_field(psi, dx, t, lam)) ** 2
    with ffx.Plan(dims, dx, t, lam, form="tc", accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        # an accumulating plan's gradient is shared by the realizations
        g1 = ffx.ffx_expand_backward(plan, to_dev(psi), to_dev(np.ascontiguousarray(grad[0]))).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(dims, dx, t, lam, form="tc") as plan:
        g = ffx.ffx_expand_backward(plan, to_dev(psi), to_dev(grad)).cpu().numpy()
        assert plan.device_errors() == 0
    e1 = rel_l2(acc, ref.sum(0))
    e2 = rel_l2(g, O.density_loss_gradient(psi, grad, dx, t, lam))
    e3 = rel_l2(g1, O.density_loss_gradient(psi, np.broadcast_to(grad[0], grad.shape), dx, t, lam))
    print(f"tc {dims}: ensemble sum {e1:.2e}, backward {e2:.2e}, shared-grad backward {e3:.2e}")
    assert e1 < DENSITY_TOL and e2 < FIELD_TOL and e3 < FIELD_TOL


@pytest.mark.parametrize("dims,lam,batch,forms", [
    ((96, 96, 96), (10, 10, 10), 1, ("tc",) * 3),       # lines of 96 points: tensor cores from one tile
    ((48, 48, 48), (20, 20, 20), 2, ("dense",) * 3),    # 36 items per pass: FP32
    ((48, 48, 48), (20, 20, 20), 4, ("tc",) * 3),       # 72 items: tensor cores
    ((1024,), (9,), 40, ("fft",)),                      # 40 lines of a 1-D plan: an FFT form
    ((1024,), (1,), 256, ("fft",)),                     # lam = 1: an FFT form beats the dense map
    ((512,), (20,), 256, ("tc",)),                      # lam = 20: tensor cores
    ((1024,), (9,), 31, ("dense",)),                    # 31 lines: the few-lines kernel
    # small lam, a large call: the lam = 1 axes take the one-term FFT kernel,
    # the lam = 2 axis the tensor cores (cheaper there than the two-term kernel)
    ((64, 64, 64), (1, 2, 1), 4, ("fft", "tc", "fft")),
    ((256, 256), (1, 2), 2, ("fft", "fft")),            # 256 points: the FFT kernels beat the dense map
    ((512,), (2,), 256, ("fft",)),                      # lam = 2 on 512 points: the FFT form stays
])
def test_auto_per_call_kernel_choice(ffx, dims, lam, batch, forms):
    rng = np.random.default_rng(sum(dims) + batch)
    dx, t = (0.25,) * len(dims), 10.0
    psi = random_field(rng, (batch,) + dims)
    with ffx.Plan(dims, dx, t, lam, fused=False) as plan:
        got = plan.call_forms(batch)
        # "fft": either FFT form (the cost model weighs paper against fold)
        assert all(g in ("fold", "paper") if f == "fft" else g == f for g, f in zip(got, forms)), got
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    e = rel_l2(rho, np.abs(O.expand_field(psi, dx, t, lam)) ** 2)
    print(f"auto {dims} x{batch} {forms}: density {e:.2e}")
    assert e < DENSITY_TOL


def test_tc_unaligned_buffers_take_the_simt_kernel(ffx):
    """A field that starts 8 bytes past a 16-byte boundary is still expanded
    correctly (those passes run on the FP32 SIMT dense kernels)."""
    dims, dx, lam, t = (128, 64), (0.25, 0.25), (3, 5), 4.0
    rng = np.random.default_rng(5)
    psi = random_field(rng, (1,) + dims)
    buf = torch.zeros(psi.size + 1, dtype=torch.complex64, device="cuda")
    view = buf[1:].view((1,) + dims)
    view.copy_(to_dev(psi))
    with ffx.Plan(dims, dx, t, lam, form="tc") as plan:
        rho = ffx.ffx_expand(plan, view).cpu().numpy()
        assert plan.device_errors() == 0
    e = rel_l2(rho, np.abs(O.expand_field(psi, dx, t, lam)) ** 2)
    print(f"tc unaligned input: density {e:.2e}")
    assert e < DENSITY_TOL


def test_auto_moves_large_dense_passes_to_tensor_cores(ffx):
    w = inputs.config_two_cloud()
    psi = w.batch_array(6)
    ref = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    with ffx.Plan(w.dims, w.dx, w.t, w.lam) as plan:
        assert plan.axis_forms == ("dense",) * 3
        assert plan.call_forms(1) == ("tc",) * 3     # batch 1: the fused launch, on the tensor cores
        assert plan.fused_max_batch == 1             # from batch 2 every pass has 64 tensor-core items
        assert plan.launches_per_call(batch=2) == 3
        assert plan.call_forms(6) == ("tc",) * 3     # 6 x 4096 lines per pass: tensor cores
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        one = ffx.ffx_expand(plan, to_dev(psi[:1])).cpu().numpy()
        assert plan.device_errors() == 0
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, form="dense") as plan:
        assert plan.call_forms(6) == ("dense",) * 3  # explicit forms never switch
    e6, e1 = rel_l2(rho, ref), rel_l2(one, ref[:1])
    print(f"auto {w.name}: batch 6 on tensor cores {e6:.2e}, batch 1 fused on tensor cores {e1:.2e}")
    assert e6 < DENSITY_TOL and e1 < DENSITY_TOL


@pytest.mark.parametrize("dims,lam,batch", [
    ((32,), (50,), 200),         # 32-point lines, two blocks per SM, a ragged last item
    ((64,), (5,), 300),          # 64-point lines, a few items per block
    ((32, 64), (7, 3), 40),      # a strided 32-point axis, then a contiguous 64-point axis
])
def test_tc_resident_passes_in_place(ffx, dims, lam, batch):
    """The passes that keep T resident and take the input operand in tensor
    memory run in place: each item reads its lines whole before it writes them."""
    rng = np.random.default_rng(sum(dims) + 3 * batch)
    dx, t = (0.25,) * len(dims), 5.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form="tc") as plan:
        assert plan.call_forms(batch) == ("tc",) * len(dims)
        x = to_dev(psi)
        ffx.ffx_expand_field(plan, x, x)
        got = x.cpu().numpy()
        assert plan.device_errors() == 0
    e = rel_l2(got, ref)
    print(f"tc in place {dims} x{batch}: field {e:.2e}")
    assert e < FIELD_TOL
