"""GPU parity of the dense form's few-lines kernel against the FP64 oracle.

Calls whose pass covers fewer than 32 lines in all (batch x lines: a 1-D
field, a handful of realizations, a thin 2-D lattice) run one warp per row of
T.  These cases cover both staged-line widths (zero padding past N), every
output kind (field, density, ensemble sum, adjoint, gradient with a shared
density gradient), strided lines, the 31/32-line switch to the tile kernels,
and in-place calls on short lines, which must keep the in-place kernel.
"""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


@pytest.mark.parametrize("N,lam,batch", [(48, 7, 1), (64, 30, 2), (96, 5, 3), (192, 11, 1), (512, 20, 1),
                                         (768, 4, 5), (1024, 9, 2), (512, 20, 31), (512, 20, 32)])
def test_1d_field_and_density(ffx, N, lam, batch):
    rng = np.random.default_rng(N + 7 * batch)
    dx, t = 0.1, 0.5 * lam
    psi = random_field(rng, (batch, N))
    ref = O.expand_field(psi, (dx,), t, (lam,))
    with ffx.Plan((N,), (dx,), t, (lam,)) as plan:
        assert plan.axis_forms == ("dense",)  # fewer than 32 lines per realization
        x = to_dev(psi)
        fld = ffx.ffx_expand_field(plan, x).cpu().numpy()
        rho = ffx.ffx_expand(plan, x).cpu().numpy()
        assert plan.device_errors() == 0
    ef, ed = rel_l2(fld, ref), rel_l2(rho, np.abs(ref) ** 2)
    print(f"N={N} lam={lam} B={batch}: field {ef:.2e} density {ed:.2e}")
    assert ef < FIELD_TOL and ed < DENSITY_TOL


@pytest.mark.parametrize("N,batch", [(64, 5), (512, 7), (1024, 3)])
def test_ensemble_sum(ffx, N, batch):
    rng = np.random.default_rng(3 * N + batch)
    dx, lam, t = 0.2, 13, 6.0
    psi = random_field(rng, (batch, N))
    ref = (np.abs(O.expand_field(psi, (dx,), t, (lam,))) ** 2).sum(axis=0)
    with ffx.Plan((N,), (dx,), t, (lam,), accumulate=True) as plan:
        out = torch.full((N,), 0.25, dtype=torch.float32, device="cuda")
        ffx.ffx_expand(plan, to_dev(psi), out)
        got = out.cpu().numpy() - 0.25
    e = rel_l2(got, ref)
    print(f"ensemble N={N} B={batch}: {e:.2e}")
    assert e < DENSITY_TOL


@pytest.mark.parametrize("dims,lam,batch", [((96, 16), (6, 3), 1),    # axis 0: 16 strided lines
                                            ((256, 16), (9, 2), 1),   # axis 0: 16 strided lines of 256
                                            ((16, 384), (3, 17), 1)])  # axis 1: 16 contiguous lines
def test_thin_2d(ffx, dims, lam, batch):
    rng = np.random.default_rng(sum(dims) + batch)
    dx, t = (0.25, 0.3), 3.0
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, form="dense") as plan:
        fld = ffx.ffx_expand_field(plan, to_dev(psi)).cpu().numpy()
    e = rel_l2(fld, ref)
    print(f"thin {dims} B={batch}: field {e:.2e}")
    assert e < FIELD_TOL


@pytest.mark.parametrize("N", [48, 512])
def test_adjoint_and_backward(ffx, N):
    rng = np.random.default_rng(N)
    dx, lam, t = 0.2, 8, 3.0
    x = random_field(rng, (2, N))
    y = random_field(rng, (2, N))
    with ffx.Plan((N,), (dx,), t, (lam,)) as plan:
        Tx = ffx.ffx_expand_field(plan, to_dev(x)).cpu().numpy()
        THy = ffx.ffx_expand_adjoint(plan, to_dev(y)).cpu().numpy()
    e = rel_l2(THy, O.expand_adjoint(y, (dx,), t, (lam,)))
    lhs = np.vdot(Tx.astype(np.complex128), y.astype(np.complex128))
    rhs = np.vdot(x.astype(np.complex128), THy.astype(np.complex128))
    assert e < FIELD_TOL
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    # gradient of an ensemble-summed density: one density gradient shared by the batch
    g = rng.normal(size=(N,)).astype(np.float32)
    with ffx.Plan((N,), (dx,), t, (lam,), accumulate=True) as plan:
        got = ffx.ffx_expand_backward(plan, to_dev(x), to_dev(g)).cpu().numpy()
    ref = O.density_loss_gradient(x, np.broadcast_to(g, (2, N)), (dx,), t, (lam,))
    eb = rel_l2(got, ref)
    print(f"N={N}: adjoint {e:.2e} backward {eb:.2e}")
    assert eb < FIELD_TOL


@pytest.mark.parametrize("N", [32, 64])
def test_in_place_short_lines(ffx, N):
    """An in-place call over a few short lines keeps the in-place kernel."""
    rng = np.random.default_rng(N + 1)
    dx, lam, t = 0.25, 10, 4.0
    psi = random_field(rng, (3, N))
    ref = O.expand_field(psi, (dx,), t, (lam,))
    with ffx.Plan((N,), (dx,), t, (lam,)) as plan:
        x = to_dev(psi)
        ffx.ffx_expand_field(plan, x, x)
        got = x.cpu().numpy()
    assert rel_l2(got, ref) < FIELD_TOL
