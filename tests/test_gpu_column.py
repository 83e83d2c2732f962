"""Detector readout on the GPU: the density integrated along one axis
(Sec. 6, ffx_expand_column) and the fringe phase of eq. dphase2
(ffx_fringe_phase), against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


# (dims, lam, batch, form, fused): the fused small-lattice launch, the per-axis
# launches (dense, FFT forms, tensor cores), contiguous and strided axes
CASES = [((64, 64, 64), (30, 30, 3), 1, "auto", True),
         ((64, 64, 64), (30, 30, 3), 3, "dense", False),
         ((32, 48), (7, 5), 2, "auto", True),
         ((48, 64, 32), (5, 7, 3), 2, "fold", False),
         ((16, 96, 32), (3, 4, 9), 1, "paper", False),
         ((128, 64), (5, 3), 2, "tc", False)]


@pytest.mark.parametrize("dims,lam,batch,form,fused", CASES)
def test_column_density_matches_oracle(ffx, dims, lam, batch, form, fused):
    rng = np.random.default_rng(sum(dims) + batch)
    dx, t = tuple(0.2 + 0.05 * j for j in range(len(dims))), 7.0
    psi = random_field(rng, (batch,) + dims)
    x = to_dev(psi)
    with ffx.Plan(dims, dx, t, lam, form=form, fused=fused) as plan:
        assert plan.fused == fused
        for axis in range(len(dims)):
            col = ffx.ffx_expand_column(plan, x, axis).cpu().numpy()
            ref = O.column_density(psi, dx, t, lam, axis)
            e = rel_l2(col, ref)
            print(f"column {dims} x{batch} {form} fused={fused} axis {axis}: {e:.2e}")
            assert col.shape == ref.shape and e < DENSITY_TOL
        assert plan.device_errors() == 0


@pytest.mark.parametrize("fused,batch", [(True, 2), (False, 3)])
def test_column_density_ensemble_sum(ffx, fused, batch):
    dims, dx, lam, t = (64, 48, 32), (0.25, 0.25, 0.3), (9, 4, 3), 5.0
    rng = np.random.default_rng(31 + batch)
    psi = random_field(rng, (batch,) + dims)
    with ffx.Plan(dims, dx, t, lam, accumulate=True, fused=fused) as plan:
        assert plan.fused == fused
        out = torch.full((64, 32), 0.5, dtype=torch.float32, device="cuda")  # added to
        ffx.ffx_expand_column(plan, to_dev(psi), 1, out)
        got = out.cpu().numpy()
    ref = 0.5 + O.column_density(psi, dx, t, lam, 1).sum(0)
    e = rel_l2(got, ref)
    print(f"column ensemble fused={fused} x{batch}: {e:.2e}")
    assert e < DENSITY_TOL


def test_fringe_readout_matches_oracle_on_the_same_image(ffx):
    """The readout takes the same decisions (peak search in float32) and the
    same FP64 refinement as the oracle's, on the very same float32 image."""
    rng = np.random.default_rng(9)
    y = -4.0 + 0.05 * np.arange(160)
    rows = []
    for r in range(97):
        y0, s_ = rng.uniform(-1, 1), rng.uniform(0.6, 2.0)
        rows.append(np.exp(-y ** 2 / 20) * np.cos(np.pi * (y - y0) / s_) ** 2 + rng.uniform(0, 1e-3, y.size))
    rows.append(np.linspace(1.0, 2.0, y.size))   # no interior maximum
    img = np.asarray(rows, dtype=np.float32)
    D, t = 2.5, 6.0
    ref = O.fringe_phase(img, y, D, t)
    for y_dim, arr in ((-1, img), (0, np.ascontiguousarray(img.T))):
        got = ffx.ffx_fringe_phase(torch.from_numpy(arr).cuda(), y[0], 0.05, D, t, y_dim=y_dim).cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert np.abs(got[ok] - ref[ok]).max() < 1e-9


def test_two_cloud_fringes_give_the_relative_phase(ffx):
    """End to end (Sec. 6): two clouds split by D along y with relative phase
    dtheta, expanded on the GPU, imaged along z, read out per x row by
    eq. dphase2; the estimate matches dtheta, and the oracle's image."""
    dims, dx, lam, t = (16, 512, 16), (0.25, 0.05, 0.25), (1, 4, 2), 6.0  # lam L = 102 along y: no wrap
    sigma, D, dtheta = 0.3, 3.0, 1.1
    xs = [O.default_a(n, d) + d * np.arange(n) for n, d in zip(dims, dx)]
    w = 1.0 / sigma ** 2
    gy = (np.exp(1j * dtheta) * np.exp(-w * (2 * xs[1] - D) ** 2 / 8)
          + np.exp(-w * (2 * xs[1] + D) ** 2 / 8))
    psi = np.einsum("i,j,k->ijk", np.exp(-xs[0] ** 2 / 8), gy, np.exp(-xs[2] ** 2 / 2))[None].astype(np.complex64)
    with ffx.Plan(dims, dx, t, lam) as plan:
        col = ffx.ffx_expand_column(plan, to_dev(psi), 2)[0]          # [x][y]
        y0, dy = ffx.output_axis(plan, 1)
        phase = ffx.ffx_fringe_phase(col, y0, dy, D, t).cpu().numpy()
    ybar = y0 + dy * np.arange(dims[1])
    ref_img = O.column_density(psi, dx, t, lam, 2)[0]
    assert rel_l2(col.cpu().numpy(), ref_img) < DENSITY_TOL
    assert np.abs(np.angle(np.exp(1j * (phase - dtheta)))).max() < 0.1
    assert np.abs(phase - O.fringe_phase(ref_img, ybar, D, t)).max() < 1e-3
