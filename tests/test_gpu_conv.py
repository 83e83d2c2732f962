"""FFT-form passes with one or two terms on lines of 16, 64, 256 and 1024
points (four-step line FFTs in registers): magnification 1 in both explicit
forms (densities, fields also in place, the adjoint and the backward pass)
and magnification 2 in the fold form, against the FP64 oracle, on contiguous
and strided axes with tiles that end inside a realization; results do not
depend on the batch a realization comes in."""

import numpy as np
import pytest

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

# (dims, batch): every axis of 16, 64 or 256 points; line counts per pass that
# are not multiples of a tile's lines (16, 32 or 64)
CASES = [
    ((64, 64, 64), 3),
    ((16, 256), 5),
    ((256, 16), 3),
    ((64, 16, 256), 1),
    ((256,), 7),
    ((1024, 16), 2),
    ((16, 1024), 3),
]


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


@pytest.mark.parametrize("form", ["fold", "paper"])
@pytest.mark.parametrize("dims,batch", CASES)
def test_conv_density_field_adjoint_backward(ffx, dims, batch, form):
    d = len(dims)
    rng = np.random.default_rng(sum(dims) + 31 * batch + (form == "paper"))
    dx = tuple(0.2 + 0.05 * j for j in range(d))
    lam, t = (1,) * d, 3.0
    psi = random_field(rng, (batch,) + dims)
    g_in = random_field(rng, (batch,) + dims)
    grad = rng.normal(size=(batch,) + dims).astype(np.float32)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form=form) as plan:
        x = to_dev(psi)
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        f = ffx.ffx_expand_field(plan, x).cpu().numpy()
        y = x.clone()
        ffx.ffx_expand_field(plan, y, y)  # in place
        adj = ffx.ffx_expand_adjoint(plan, to_dev(g_in)).cpu().numpy()
        gb = ffx.ffx_expand_backward(plan, x, to_dev(grad)).cpu().numpy()
        assert plan.device_errors() == 0
    e_d = rel_l2(rho, np.abs(ref) ** 2)
    e_f = rel_l2(f, ref)
    e_a = rel_l2(adj, O.expand_adjoint(g_in, dx, t, lam))
    e_g = rel_l2(gb, O.density_loss_gradient(psi, grad, dx, t, lam))
    print(f"conv {form} {dims} x{batch}: density {e_d:.2e}, field {e_f:.2e}, adjoint {e_a:.2e}, backward {e_g:.2e}")
    assert e_d < DENSITY_TOL and e_f < FIELD_TOL and e_a < FIELD_TOL and e_g < FIELD_TOL
    assert np.array_equal(y.cpu().numpy(), f)


def test_conv_batch_independent_bitwise(ffx):
    dims, lam, dx, t = (64, 256), (1, 1), (0.25, 0.25), 2.0
    psi = random_field(np.random.default_rng(5), (6,) + dims)
    with ffx.Plan(dims, dx, t, lam, form="fold") as plan:
        all6 = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        one = ffx.ffx_expand(plan, to_dev(psi[4:5])).cpu().numpy()
    assert np.array_equal(all6[4:5], one)


# magnification 2 (two terms folded into one spectrum), fold form
CASES_LAM2 = [
    ((64, 64, 64), 2),
    ((256, 16), 3),
    ((16, 1024), 2),
    ((1024,), 5),
]


@pytest.mark.parametrize("dims,batch", CASES_LAM2)
def test_conv_two_terms_fold(ffx, dims, batch):
    d = len(dims)
    rng = np.random.default_rng(sum(dims) + 7 * batch)
    dx = tuple(0.25 - 0.02 * j for j in range(d))
    lam, t = (2,) * d, 5.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form="fold") as plan:
        x = to_dev(psi)
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        f = ffx.ffx_expand_field(plan, x).cpu().numpy()
        y = x.clone()
        ffx.ffx_expand_field(plan, y, y)
        assert plan.device_errors() == 0
    e_d, e_f = rel_l2(rho, np.abs(ref) ** 2), rel_l2(f, ref)
    print(f"conv lam 2 fold {dims} x{batch}: density {e_d:.2e}, field {e_f:.2e}")
    assert e_d < DENSITY_TOL and e_f < FIELD_TOL
    assert np.array_equal(y.cpu().numpy(), f)
