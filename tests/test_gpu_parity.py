"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: relative L2 density error <= 2e-5 against FP64 (and the same for the
complex field), on the same seeded inputs (complex64, promoted to complex128
for the oracle).  Sizes span several tiles and ragged tails; the full-size
workloads are checked on sampled lines the oracle computes one by one.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1602_03395_gb300 import inputs
from gpu_common import (DENSITY_TOL, FIELD_TOL, gpu_density, gpu_field, random_field,
                        rel_l2, require_gpu, to_dev)

pytestmark = pytest.mark.gpu

LENGTHS = [16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 2048]


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


@pytest.mark.parametrize("form", ["paper", "fold", "dense"])
@pytest.mark.parametrize("N", LENGTHS)
def test_1d_every_length(ffx, N, form):
    if form == "dense" and N > 1024:
        pytest.skip("the dense form takes lines up to 1024 points")
    rng = np.random.default_rng(N)
    for lam, t in [(1, 0.7), (3, 2.0), (8, 5.0)]:
        if form == "paper" and N >= 1024 and lam == 8:
            lam = 5
        dx = 0.2
        psi = random_field(rng, (3, N))
        ref = O.expand_field(psi, (dx,), t, (lam,))
        got = gpu_field(ffx, psi, (N,), (dx,), t, (lam,), form=form)
        ef = rel_l2(got, ref)
        rho = gpu_density(ffx, psi, (N,), (dx,), t, (lam,), form=form)
        ed = rel_l2(rho, np.abs(ref) ** 2)
        print(f"N={N} lam={lam} form={form}: field {ef:.2e} density {ed:.2e}")
        assert ef < FIELD_TOL and ed < DENSITY_TOL


@pytest.mark.parametrize("form", ["paper", "fold", "dense"])
@pytest.mark.parametrize("N,lam", [(16, 100), (64, 64), (32, 50), (48, 36), (96, 30), (128, 100)])
def test_large_magnification_and_common_factors(ffx, N, lam, form):
    """lam > N (q wraps modulo N in the fold) and gcd(lam, N) large (several
    fine indices fold onto one bin)."""
    rng = np.random.default_rng(lam * 1000 + N)
    dx, t = 0.25, 4.0 * lam
    psi = random_field(rng, (2, N))
    ref = O.expand_field(psi, (dx,), t, (lam,))
    got = gpu_field(ffx, psi, (N,), (dx,), t, (lam,), form=form)
    e = rel_l2(got, ref)
    print(f"N={N} lam={lam} form={form}: field {e:.2e}")
    assert e < FIELD_TOL


@pytest.mark.parametrize("frac", [0.0, 0.37, 0.5])
def test_offsets(ffx, frac):
    """Custom input offset and non-integer output offsets (s = (abar-a)/dx)."""
    N, lam, dx, t = 128, 7, 0.15, 3.0
    a = -3.1
    abar = a - (300 + frac) * dx
    rng = np.random.default_rng(3)
    psi = random_field(rng, (N,))
    ref = O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    for form in ("paper", "fold", "dense"):
        got = gpu_field(ffx, psi, (N,), (dx,), t, (lam,), form=form, a=(a,), abar=(abar,))
        assert rel_l2(got, ref) < FIELD_TOL


def test_t0_is_subsampling(ffx):
    N, lam, dx = 64, 4, 0.3
    rng = np.random.default_rng(0)
    psi = random_field(rng, (N,))
    got = gpu_field(ffx, psi, (N,), (dx,), 0.0, (lam,))
    s = -((lam - 1) * N) // 2
    idx = np.mod(s + lam * np.arange(N), lam * N)
    ex = np.where(idx < N, psi[np.minimum(idx, N - 1)], 0)
    assert np.abs(got - ex).max() < 1e-5 * np.abs(psi).max()


@pytest.mark.parametrize("form", ["paper", "fold", "dense", "auto"])
@pytest.mark.parametrize("dims,lam,batch", [
    ((48, 64), (5, 3), 1),           # ragged tiles on both axes
    ((96, 32), (2, 9), 3),
    ((16, 32, 48), (3, 4, 2), 2),
    ((64, 16, 96), (6, 1, 5), 1),
    ((32, 48, 16), (11, 3, 7), 3),
    ((128, 16, 256), (9, 2, 5), 2),  # dense passes over 64 points run out of place
])
def test_nd_batches(ffx, dims, lam, batch, form):
    rng = np.random.default_rng(sum(dims) + batch)
    dx = tuple(0.2 + 0.03 * j for j in range(len(dims)))
    t = 2.5
    psi = random_field(rng, (batch,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    got = gpu_field(ffx, psi, dims, dx, t, lam, form=form)
    rho = gpu_density(ffx, psi, dims, dx, t, lam, form=form)
    ef, ed = rel_l2(got, ref), rel_l2(rho, np.abs(ref) ** 2)
    print(f"dims={dims} lam={lam} B={batch} {form}: field {ef:.2e} density {ed:.2e}")
    assert ef < FIELD_TOL and ed < DENSITY_TOL


@pytest.mark.parametrize("form", ["fold", "dense"])
def test_accumulate(ffx, form):
    dims, dx, lam, t = (32, 16, 64), (0.25, 0.3, 0.2), (4, 3, 5), 3.0
    rng = np.random.default_rng(12)
    psi = random_field(rng, (5,) + dims)
    ref = (np.abs(O.expand_field(psi, dx, t, lam)) ** 2).sum(axis=0)
    plan = ffx.Plan(dims, dx, t, lam, accumulate=True, form=form)
    out = torch.full(dims, 0.5, dtype=torch.float32, device="cuda")
    ffx.ffx_expand(plan, to_dev(psi), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy() - 0.5
    plan.close()
    e = rel_l2(got, ref)
    print(f"accumulate: {e:.2e}")
    assert e < DENSITY_TOL


def test_determinism_and_batch_independence(ffx):
    dims, dx, lam, t = (48, 64, 32), (0.25,) * 3, (5, 7, 3), 6.0
    rng = np.random.default_rng(21)
    psi = random_field(rng, (3,) + dims)
    plan = ffx.Plan(dims, dx, t, lam)
    x = to_dev(psi)
    a1 = ffx.ffx_expand(plan, x).cpu()
    a2 = ffx.ffx_expand(plan, x).cpu()
    single = ffx.ffx_expand(plan, x[1:2].contiguous()).cpu()
    plan.close()
    assert torch.equal(a1, a2)
    assert torch.equal(a1[1:2], single)


# ---------------------------------------------------------------------------
# the workloads at full size
# ---------------------------------------------------------------------------

def test_workload_1d_tf_solitons(ffx):
    w = inputs.config_1d()
    psi = w.batch_array()
    ref = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    for form in ("paper", "fold", "dense"):
        got = gpu_density(ffx, psi, w.dims, w.dx, w.t, w.lam, form=form)
        e = rel_l2(got, ref)
        print(f"{w.name} {form}: density rel L2 {e:.2e}")
        assert e < DENSITY_TOL


def test_workload_two_cloud_64(ffx):
    w = inputs.config_two_cloud()
    psi = w.batch_array()
    ref = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    for form in ("paper", "fold", "dense", "auto"):
        got = gpu_density(ffx, psi, w.dims, w.dx, w.t, w.lam, form=form)
        e = rel_l2(got, ref)
        print(f"{w.name} {form}: density rel L2 {e:.2e}")
        assert e < DENSITY_TOL


def test_workload_quasicondensate_full_batch(ffx):
    """The quasicondensate ensemble at its full size, 256 realizations of
    32x32x512 in one call, as the benchmark runs it: a seeded sample of 8
    realizations element by element against the FP64 oracle (worst one held
    to the bar), and the ensemble mean of an accumulating call against the
    oracle's mean over all 256."""
    w = inputs.config_quasicondensate()
    assert w.batch == 256
    psi = w.batch_array()
    x = to_dev(psi)
    with ffx.Plan(w.dims, w.dx, w.t, w.lam) as plan:
        rho = ffx.ffx_expand(plan, x)
        torch.cuda.synchronize()
        assert plan.device_errors() == 0
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, accumulate=True) as plan:
        acc = ffx.ffx_expand(plan, x).cpu().numpy()
    sample = sorted(np.random.default_rng(256).choice(w.batch, size=8, replace=False).tolist())
    worst = 0.0
    for b in sample:
        ref = np.abs(O.expand_field(psi[b], w.dx, w.t, w.lam)) ** 2
        worst = max(worst, rel_l2(rho[b].cpu().numpy(), ref))
    mean = np.zeros(w.dims)
    for b0 in range(0, w.batch, 32):
        mean += (np.abs(O.expand_field(psi[b0:b0 + 32], w.dx, w.t, w.lam)) ** 2).sum(0)
    mean /= w.batch
    e_mean = rel_l2(acc / w.batch, mean)
    print(f"{w.name} x{w.batch}: worst of 8 sampled realizations {worst:.2e}, ensemble mean {e_mean:.2e}")
    assert worst < DENSITY_TOL and e_mean < DENSITY_TOL


@pytest.mark.parametrize("form", ["auto", "fold"])
def test_workload_quasicondensate_ensemble(ffx, form):
    w = inputs.config_quasicondensate(batch=4)
    psi = w.batch_array()
    per = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    got = gpu_density(ffx, psi, w.dims, w.dx, w.t, w.lam, form=form)
    worst = max(rel_l2(got[b], per[b]) for b in range(w.batch))
    acc = gpu_density(ffx, psi, w.dims, w.dx, w.t, w.lam, accumulate=True, form=form)
    e_mean = rel_l2(acc / w.batch, per.mean(axis=0))
    print(f"{w.name}: worst realization {worst:.2e}, ensemble mean {e_mean:.2e}")
    assert worst < DENSITY_TOL and e_mean < DENSITY_TOL


@pytest.mark.parametrize("form", ["auto", "fold"])
@pytest.mark.parametrize("which", ["two_cloud", "quasicondensate"])
def test_workload_large_sampled_lines(ffx, which, form):
    """256^3 / 128x128x1024 with lam = 100 on every axis: output lines computed
    one by one by the oracle.  Lines through the bright centre of the image
    (the magnified box is centred on the input box) are held to the 2e-5
    relative L2 bar, pooled; lines at random positions, mostly in the dark
    wings where densities are ~1e-20 of the peak, to 2e-5 of the peak."""
    w = inputs.config_large(which)
    psi = w.realization(0)
    plan = ffx.Plan(w.dims, w.dx, w.t, w.lam, form=form)
    forms = plan.axis_forms
    rho = ffx.ffx_expand(plan, to_dev(psi[None])).cpu().numpy()[0]
    plan.close()
    rng = np.random.default_rng(99)
    d = len(w.dims)
    num = den = 0.0
    worst_abs = 0.0
    peak = rho.max()
    for axis in range(d):
        for kind in ("centre", "centre", "random"):
            if kind == "centre":
                index = tuple(w.dims[j] // 2 + int(rng.integers(-2, 3)) for j in range(d) if j != axis)
            else:
                index = tuple(int(rng.integers(0, w.dims[j])) for j in range(d) if j != axis)
            ref = np.abs(O.sample_lines(psi, w.dx, w.t, w.lam, axis, index)) ** 2
            sl = list(index)
            sl.insert(axis, slice(None))
            got = rho[tuple(sl)]
            if kind == "centre":
                num += np.sum((got - ref) ** 2)
                den += np.sum(ref ** 2)
            worst_abs = max(worst_abs, np.abs(got - ref).max())
    pooled = np.sqrt(num / den)
    print(f"{w.name} {forms}: centre lines pooled rel L2 {pooled:.2e}; worst abs error / peak "
          f"{worst_abs / peak:.2e}")
    assert pooled < DENSITY_TOL
    assert worst_abs < DENSITY_TOL * peak


# ---------------------------------------------------------------------------
# adjoint and gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", ["fold", "dense"])
@pytest.mark.parametrize("dims,lam", [((64,), (9,)), ((48, 32), (4, 6)), ((16, 32, 64), (3, 5, 2)),
                                      ((128, 96), (7, 3))])
def test_adjoint_against_oracle_and_dot_product(ffx, dims, lam, form):
    rng = np.random.default_rng(len(dims) * 7)
    dx = (0.25,) * len(dims)
    t = 3.0
    x = random_field(rng, (2,) + dims)
    y = random_field(rng, (2,) + dims)
    plan = ffx.Plan(dims, dx, t, lam, form=form)
    Tx = ffx.ffx_expand_field(plan, to_dev(x)).cpu().numpy()
    THy = ffx.ffx_expand_adjoint(plan, to_dev(y)).cpu().numpy()
    plan.close()
    ref = O.expand_adjoint(y, dx, t, lam)
    e = rel_l2(THy, ref)
    lhs = np.vdot(Tx.astype(np.complex128), y.astype(np.complex128))
    rhs = np.vdot(x.astype(np.complex128), THy.astype(np.complex128))
    print(f"adjoint dims={dims}: vs oracle {e:.2e}, dot-product gap {abs(lhs - rhs) / abs(lhs):.2e}")
    assert e < FIELD_TOL
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


@pytest.mark.parametrize("form", ["fold", "dense"])
@pytest.mark.parametrize("dims", [(32, 48, 16), (128, 16, 96)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_backward_against_oracle(ffx, accumulate, dims, form):
    dx, lam, t = (0.25, 0.2, 0.3), (5, 3, 4), 2.0
    rng = np.random.default_rng(5)
    psi = random_field(rng, (3,) + dims)
    gshape = dims if accumulate else (3,) + dims
    grad = rng.normal(size=gshape).astype(np.float32)
    plan = ffx.Plan(dims, dx, t, lam, accumulate=accumulate, form=form)
    got = ffx.ffx_expand_backward(plan, to_dev(psi), to_dev(grad)).cpu().numpy()
    plan.close()
    gfull = np.broadcast_to(grad, (3,) + dims)
    ref = O.density_loss_gradient(psi, gfull, dx, t, lam)
    e = rel_l2(got, ref)
    print(f"backward acc={accumulate} dims={dims} {form}: {e:.2e}")
    assert e < FIELD_TOL


def test_autograd_gradient_finite_differences(ffx):
    """Gradient of L = sum (rho - target)^2 via the autograd front end, checked
    against central finite differences of the FP64 oracle's loss on 16 seeded
    directions."""
    dims, dx, lam, t = (16, 32, 48), (0.3, 0.25, 0.2), (3, 4, 2), 1.5
    rng = np.random.default_rng(16)
    psi = random_field(rng, dims)
    target = (np.abs(O.expand_field(random_field(rng, dims), dx, t, lam)) ** 2).astype(np.float32)
    plan = ffx.Plan(dims, dx, t, lam)
    x = to_dev(psi[None]).requires_grad_(True)
    rho = ffx.expand_density(x, plan)
    loss = ((rho - to_dev(target[None])) ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy()[0].astype(np.complex128)
    plan.close()

    def L(p):
        return np.sum((O.expand_density(p, dx, t, lam) - target) ** 2)

    p64 = psi.astype(np.complex128)
    worst = 0.0
    for i in range(16):
        v = rng.normal(size=dims) + 1j * rng.normal(size=dims)
        eps = 1e-4 * np.linalg.norm(p64) / np.linalg.norm(v)
        fd = (L(p64 + eps * v) - L(p64 - eps * v)) / (2 * eps)
        an = np.real(np.vdot(g, v))
        worst = max(worst, abs(fd - an) / max(abs(fd), 1e-30))
    print(f"FD worst relative gap {worst:.2e}")
    assert worst < 1e-4


def test_large_adjoint_and_gradient_properties(ffx):
    """256^3, lam = 100: the dot-product identity <T x, y> = <x, T^H y> at full
    size, and <grad, v> against central differences of the GPU loss (FP32
    densities, loss summed in FP64) on 16 seeded directions v shaped like the
    cloud."""
    w = inputs.config_large("two_cloud")
    psi = to_dev(w.realization(0)[None])
    plan = ffx.Plan(w.dims, w.dx, w.t, w.lam)
    target = ffx.ffx_expand(plan, to_dev(w.realization(1)[None]))
    gen = torch.Generator(device="cuda").manual_seed(1234)
    y = torch.randn(psi.shape, dtype=torch.complex64, device="cuda", generator=gen)
    Tx = ffx.ffx_expand_field(plan, psi)
    THy = ffx.ffx_expand_adjoint(plan, y)
    lhs = torch.vdot(Tx.flatten().to(torch.complex128), y.flatten().to(torch.complex128)).item()
    rhs = torch.vdot(psi.flatten().to(torch.complex128), THy.flatten().to(torch.complex128)).item()
    gap = abs(lhs - rhs) / abs(lhs)

    def loss(p):
        r = ffx.ffx_expand(plan, p)
        return ((r.double() - target.double()) ** 2).sum().item()

    rho = ffx.ffx_expand(plan, psi)
    g = ffx.ffx_expand_backward(plan, psi, (2 * (rho - target)).contiguous())
    worst = 0.0
    # directions psi * (c0 + c . x / L) with seeded complex c: perturbations of the
    # cloud whose effect on L is O(L) (a white-noise direction has <grad, v> ~
    # L / sqrt(points), drowned by the FP32 noise of the loss)
    coords = [torch.linspace(-0.5, 0.5, n, device="cuda") for n in w.dims]
    X, Y, Z = torch.meshgrid(*coords, indexing="ij")
    for i in range(16):
        c = torch.randn(4, dtype=torch.complex64, device="cuda", generator=gen)
        v = (psi * (c[0] + c[1] * X + c[2] * Y + c[3] * Z)).contiguous()
        eps = 1e-2 * psi.abs().pow(2).sum().sqrt().item() / v.abs().pow(2).sum().sqrt().item()

        def dq(e):
            return (loss(psi + e * v) - loss(psi - e * v)) / (2 * e)

        # Richardson: the O(eps^2) truncation of the central difference cancels,
        # and eps stays large against the ~1e-7 relative noise of FP32 densities
        fd = (4 * dq(eps) - dq(2 * eps)) / 3
        an = (g.conj() * v).real.double().sum().item()
        worst = max(worst, abs(fd - an) / abs(fd))
    plan.close()
    print(f"large: dot-product gap {gap:.2e}, FD worst relative gap {worst:.2e}")
    assert gap < 1e-5
    assert worst < 2e-3


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_empty_batch_and_errors(ffx):
    plan = ffx.Plan((64,), (0.2,), 1.0, (3,))
    empty = torch.empty((0, 64), dtype=torch.complex64, device="cuda")
    out = torch.empty((0, 64), dtype=torch.float32, device="cuda")
    assert ffx.ffx_expand(plan, empty, out).shape == (0, 64)
    plan.close()
    with pytest.raises(ffx.FfxError) as ei:
        ffx.Plan((100,), (0.2,), 1.0, (3,))
    assert ei.value.code == ffx.FFX_EUNSUPPORTED
    with pytest.raises(ffx.FfxError) as ei:
        ffx.Plan((64,), (0.2,), 1.0, (0,))
    assert ei.value.code == ffx.FFX_EINVAL
    with pytest.raises(ffx.FfxError) as ei:
        ffx.Plan((64,), (-0.2,), 1.0, (2,))
    assert ei.value.code == ffx.FFX_EINVAL
    # misaligned device pointer
    lib = ffx.load_library()
    plan = ffx.Plan((64,), (0.2,), 1.0, (3,))
    buf = torch.zeros(130, dtype=torch.float32, device="cuda")
    import ctypes
    rc = lib.ffx_expand(plan.handle, ctypes.c_void_p(buf.data_ptr() + 4), 1,
                        ctypes.c_void_p(buf.data_ptr()), None)
    assert rc == ffx.FFX_EINVAL
    plan.close()


def test_in_place_field_with_out_of_place_passes(ffx):
    """Dense passes over lines longer than 64 points cannot run in place; an
    in-place ffx_expand_field still returns the right field."""
    dims, dx, lam, t = (128, 32, 256), (0.2, 0.25, 0.15), (6, 4, 9), 2.0
    rng = np.random.default_rng(31)
    psi = random_field(rng, (2,) + dims)
    ref = O.expand_field(psi, dx, t, lam)
    plan = ffx.Plan(dims, dx, t, lam, form="dense")
    x = to_dev(psi)
    ffx.ffx_expand_field(plan, x, x)
    got = x.cpu().numpy()
    y = to_dev(psi)
    back = ffx.ffx_expand_adjoint(plan, y, y).cpu().numpy()
    plan.close()
    assert rel_l2(got, ref) < FIELD_TOL
    assert rel_l2(back, O.expand_adjoint(psi, dx, t, lam)) < FIELD_TOL


def test_tuner_times_forms_and_caches(ffx, tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("FFX_TUNE_CACHE", str(cache))
    dims, dx, lam, t = (64, 48, 128), (0.25,) * 3, (20, 3, 2), 10.0
    p1 = ffx.Plan(dims, dx, t, lam, tune=True)
    forms = p1.axis_forms
    p1.close()
    lines = cache.read_text().splitlines()
    assert len(lines) == 3 and all('"ms": [' in ln for ln in lines)
    p2 = ffx.Plan(dims, dx, t, lam)  # reads the cache
    assert p2.axis_forms == forms
    rng = np.random.default_rng(2)
    psi = random_field(rng, (1,) + dims)
    got = ffx.ffx_expand(p2, to_dev(psi)).cpu().numpy()
    p2.close()
    ref = np.abs(O.expand_field(psi, dx, t, lam)) ** 2
    print(f"tuned forms {forms}: density {rel_l2(got, ref):.2e}")
    assert rel_l2(got, ref) < DENSITY_TOL
