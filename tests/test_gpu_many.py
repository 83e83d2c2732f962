"""Many-instance plans: uneven lattices, magnifications and flight times in
one persistent launch per axis pass, replayed as a CUDA graph.  Every
instance against the FP64 oracle and against its own single-lattice plan."""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev
from paper_1602_03395_gb300 import inputs

pytestmark = pytest.mark.gpu


def mixed_specs(count, seed=4, lam_max=12, dims_override=None):
    ws = inputs.config_mixed_batch(seed=seed, count=count)
    specs, psis = [], []
    rng = np.random.default_rng(seed)
    for i, w in enumerate(ws):
        dims = dims_override[i % len(dims_override)] if dims_override else w.dims
        lam = int(rng.integers(2, lam_max + 1))
        specs.append((dims, w.dx[:len(dims)], 4.0 * lam, (lam,) * len(dims)))
        psis.append(random_field(rng, dims) if dims_override else w.realization(0))
    return specs, psis


def pack(plan, psis):
    x = np.zeros(plan.points, np.complex64)
    for off, p in zip(plan.offsets, psis):
        x[off:off + p.size] = p.ravel()
    return x


@pytest.mark.parametrize("form", ["fold", "paper", "dense"])
def test_many_mixed_shapes_against_oracle(form):
    ffx = require_gpu()
    dims_set = [(48, 16, 32), (32, 32), (96,), (16, 128, 16), (64, 48, 16), (192, 16)]
    specs, psis = mixed_specs(9, dims_override=dims_set)
    plan = ffx.PlanMany(specs, form=form)
    x = to_dev(pack(plan, psis))
    rho = ffx.ffx_expand(plan, x).cpu().numpy()
    field = ffx.ffx_expand_field(plan, x).cpu().numpy()
    worst_d = worst_f = 0.0
    for (dims, dx, t, lam), p, off in zip(specs, psis, plan.offsets):
        ref = O.expand_field(p, dx, t, lam)
        m = p.size
        worst_d = max(worst_d, rel_l2(rho[off:off + m].reshape(dims), np.abs(ref) ** 2))
        worst_f = max(worst_f, rel_l2(field[off:off + m].reshape(dims), ref))
    plan.close()
    print(f"many ({form}): worst density {worst_d:.2e}, worst field {worst_f:.2e}")
    assert worst_d < DENSITY_TOL and worst_f < FIELD_TOL


TC_DIMS = [(48, 32, 32), (32, 32), (96,), (64, 128, 32), (64, 48, 32), (192, 32)]


@pytest.mark.parametrize("tf32", [False, True])
def test_many_tc_against_oracle(tf32):
    """Tensor-core phases: every line length a multiple of 16 from 32,
    narrower last row blocks (48, 96, 192), strided and contiguous axes, 1-D
    to 3-D instances.  By default every pass runs on the BF16 kernel (the
    48-, 96- and 192-point axes end on a half K chunk); tf32 keeps split TF32
    throughout."""
    ffx = require_gpu()
    specs, psis = mixed_specs(9, dims_override=TC_DIMS)
    plan = ffx.PlanMany(specs, form="tc", tf32=tf32)
    assert plan.form == "tc"
    assert plan.bf16 == (not tf32)
    x = to_dev(pack(plan, psis))
    rho = ffx.ffx_expand(plan, x).cpu().numpy()
    field = ffx.ffx_expand_field(plan, x).cpu().numpy()
    assert plan.device_errors() == 0
    worst_d = worst_f = 0.0
    for (dims, dx, t, lam), p, off in zip(specs, psis, plan.offsets):
        ref = O.expand_field(p, dx, t, lam)
        m = p.size
        worst_d = max(worst_d, rel_l2(rho[off:off + m].reshape(dims), np.abs(ref) ** 2))
        worst_f = max(worst_f, rel_l2(field[off:off + m].reshape(dims), ref))
    plan.close()
    print(f"many (tc, tf32={tf32}): worst density {worst_d:.2e}, worst field {worst_f:.2e}")
    assert worst_d < DENSITY_TOL and worst_f < FIELD_TOL


@pytest.mark.parametrize("tf32", [False, True])
def test_many_tc_backward_against_oracle(tf32):
    """Backward calls: the first adjoint pass (with the gradient factors) on
    split TF32 and the others on BF16 in the same phase by default."""
    ffx = require_gpu()
    specs, psis = mixed_specs(5, dims_override=[(32, 48), (48, 32, 32), (64,), (96, 32), (128, 32)])
    plan = ffx.PlanMany(specs, form="tc", tf32=tf32)
    assert plan.form == "tc"
    rng = np.random.default_rng(8)
    grads = [rng.normal(size=p.shape).astype(np.float32) for p in psis]
    g = np.zeros(plan.points, np.float32)
    for off, gr in zip(plan.offsets, grads):
        g[off:off + gr.size] = gr.ravel()
    got = ffx.ffx_expand_backward(plan, to_dev(pack(plan, psis)), to_dev(g)).cpu().numpy()
    assert plan.device_errors() == 0
    worst = 0.0
    for (dims, dx, t, lam), p, gr, off in zip(specs, psis, grads, plan.offsets):
        ref = O.density_loss_gradient(p, gr, dx, t, lam)
        worst = max(worst, rel_l2(got[off:off + p.size].reshape(dims), ref))
    plan.close()
    print(f"many backward (tc, tf32={tf32}): worst {worst:.2e}")
    assert worst < FIELD_TOL


def test_many_tc_falls_back_for_16_point_lines():
    """A 16-point axis has no tensor-core tile: the tc form keeps the FP32
    dense phases for the whole plan."""
    ffx = require_gpu()
    with ffx.PlanMany([((16, 32), (0.2, 0.2), 3.0, (5, 5)), ((64,), (0.1,), 2.0, (9,))], form="tc") as plan:
        assert plan.form == "dense"


def test_many_workload_shapes_match_single_plans_and_replay():
    """Instances of the mixed-batch workload (48^3, 64^3, 96^3, 128x32x32) with
    moderate lam: each equals its own single-lattice plan; a second call with
    new buffers (graph parameter update) gives the same result."""
    ffx = require_gpu()
    specs, psis = mixed_specs(8, lam_max=10)
    plan = ffx.PlanMany(specs)
    x = to_dev(pack(plan, psis))
    r1 = ffx.ffx_expand(plan, x).clone()
    x2 = x.clone()
    r2 = ffx.ffx_expand(plan, x2)
    assert torch.equal(r1, r2)
    r1 = r1.cpu().numpy()
    worst = 0.0
    for (dims, dx, t, lam), p, off in zip(specs, psis, plan.offsets):
        with ffx.Plan(dims, dx, t, lam) as single:
            ref = ffx.ffx_expand(single, to_dev(p[None])).cpu().numpy()[0]
        worst = max(worst, rel_l2(r1[off:off + p.size].reshape(dims), ref))
    plan.close()
    print(f"many vs single plans: worst {worst:.2e}")
    assert worst < 1e-5


@pytest.mark.parametrize("form", ["auto", "dense"])
def test_many_backward_against_oracle(form):
    ffx = require_gpu()
    dims_set = [(32, 48), (16, 32, 16), (64,), (96, 16)]
    specs, psis = mixed_specs(4, dims_override=dims_set)
    plan = ffx.PlanMany(specs, form=form)
    rng = np.random.default_rng(3)
    grads = [rng.normal(size=p.shape).astype(np.float32) for p in psis]
    g = np.zeros(plan.points, np.float32)
    for off, gr in zip(plan.offsets, grads):
        g[off:off + gr.size] = gr.ravel()
    got = ffx.ffx_expand_backward(plan, to_dev(pack(plan, psis)), to_dev(g)).cpu().numpy()
    worst = 0.0
    for (dims, dx, t, lam), p, gr, off in zip(specs, psis, grads, plan.offsets):
        ref = O.density_loss_gradient(p, gr, dx, t, lam)
        worst = max(worst, rel_l2(got[off:off + p.size].reshape(dims), ref))
    plan.close()
    print(f"many backward ({form}): worst {worst:.2e}")
    assert worst < FIELD_TOL


def test_many_rejects_unsupported():
    ffx = require_gpu()
    with pytest.raises(ffx.FfxError) as ei:
        ffx.PlanMany([((512,), (0.1,), 1.0, (3,))])
    assert ei.value.code == ffx.FFX_EUNSUPPORTED


@pytest.mark.parametrize("form", ["auto", "dense"])
def test_many_dense_auto_on_the_mixed_workload(form):
    """The mixed-batch workload's magnifications (10..100) make the dense maps
    cheaper than the fold form on every axis: the automatic form takes them,
    on the tensor cores (every line length is a multiple of 16 from 32);
    instances against the oracle, field in place, and a replay with new
    buffers."""
    ffx = require_gpu()
    ws = inputs.config_mixed_batch(count=6)
    specs = [(w.dims, w.dx, w.t, w.lam) for w in ws]
    psis = [w.realization(0) for w in ws]
    plan = ffx.PlanMany(specs, form=form)
    assert plan.form == ("tc" if form == "auto" else "dense")
    x = to_dev(pack(plan, psis))
    rho = ffx.ffx_expand(plan, x).cpu().numpy()
    y = x.clone()
    ffx.ffx_expand_field(plan, y, y)
    field = y.cpu().numpy()
    worst_d = worst_f = 0.0
    for (dims, dx, t, lam), p, off in zip(specs, psis, plan.offsets):
        ref = O.expand_field(p, dx, t, lam)
        m = p.size
        worst_d = max(worst_d, rel_l2(rho[off:off + m].reshape(dims), np.abs(ref) ** 2))
        worst_f = max(worst_f, rel_l2(field[off:off + m].reshape(dims), ref))
    r2 = ffx.ffx_expand(plan, x.clone()).cpu().numpy()
    assert plan.device_errors() == 0
    plan.close()
    print(f"many {plan.form} ({form}) on the workload: worst density {worst_d:.2e}, field {worst_f:.2e}")
    assert worst_d < DENSITY_TOL and worst_f < FIELD_TOL
    assert np.array_equal(r2, rho)


def test_many_dense_in_place_guard():
    ffx = require_gpu()
    plan = ffx.PlanMany([((96,), (0.1,), 1.0, (40,)), ((32, 32), (0.2, 0.2), 2.0, (30, 30))], form="dense")
    x = to_dev(np.ones(plan.points, np.complex64))
    with pytest.raises(ffx.FfxError) as ei:
        ffx.ffx_expand_field(plan, x, x)
    assert ei.value.code == ffx.FFX_EUNSUPPORTED
    plan.close()


def test_many_full_mixed_workload_sampled_instances():
    """The whole mixed-batch workload: 1000 instances over 48^3, 64^3, 96^3 and
    128x32x32 with lam ~ U{10..100} and t = 4 lam, in one many-instance plan
    (one persistent launch per axis phase over about 450 distinct operand
    geometries).  Forty instances are compared element by element with the FP64
    oracle: every lattice shape's smallest and largest magnification, and a
    seeded sample spread over the instance list (and so over the cost-sorted
    work list: early, middle and late items).  The other instances carry copies
    of one realization per shape: their values do not change the work."""
    ffx = require_gpu()
    ws = inputs.config_mixed_batch(count=1000)
    specs = [(w.dims, w.dx, w.t, w.lam) for w in ws]
    plan = ffx.PlanMany(specs)
    chosen = set()
    for shape in inputs.MIXED_SHAPES:
        idx = [i for i, w in enumerate(ws) if tuple(w.dims) == shape]
        chosen.add(min(idx, key=lambda i: ws[i].lam[0]))
        chosen.add(max(idx, key=lambda i: ws[i].lam[0]))
    rng = np.random.default_rng(40)
    rest = [i for i in range(len(ws)) if i not in chosen]
    for part in np.array_split(np.array(rest), 32):
        chosen.add(int(rng.choice(part)))
    chosen = sorted(chosen)
    x = torch.empty(plan.points, dtype=torch.complex64, device="cuda")
    views = plan.unpack(x)
    filler, own = {}, {}
    for i, w in enumerate(ws):
        if i in chosen:
            own[i] = w.realization(0)
            views[i].copy_(torch.from_numpy(own[i]))
        else:
            key = tuple(w.dims)
            if key not in filler:
                filler[key] = torch.from_numpy(w.realization(1)).cuda()
            views[i].copy_(filler[key])
    rho = ffx.ffx_expand(plan, x)
    torch.cuda.synchronize()
    assert plan.device_errors() == 0
    form = plan.form
    out = plan.unpack(rho)
    worst, geoms = 0.0, set()
    for i in chosen:
        w = ws[i]
        ref = np.abs(O.expand_field(own[i], w.dx, w.t, w.lam)) ** 2
        got = out[i].cpu().numpy()
        worst = max(worst, rel_l2(got, ref))
        geoms.add((tuple(w.dims), w.lam[0]))
    plan.close()
    print(f"many full workload ({form}): {len(chosen)} instances, {len(geoms)} geometries, "
          f"worst density {worst:.2e}")
    assert len(chosen) >= 40
    assert worst < DENSITY_TOL


def test_many_bf16_phases_match_tf32_phases_and_are_batch_independent():
    """The BF16 phases on the mixed-batch shapes (48^3, 64^3, 96^3,
    128x32x32): every instance within the density tolerance of the split-TF32
    plan's, and
    an instance's densities do not depend on the other instances in the plan
    (bitwise: its items run the same arithmetic wherever they are dealt)."""
    ffx = require_gpu()
    ws = inputs.config_mixed_batch(count=12)
    specs = [(w.dims, w.dx, w.t, w.lam) for w in ws]
    psis = [w.realization(0) for w in ws]
    with ffx.PlanMany(specs) as pb, ffx.PlanMany(specs, tf32=True) as pt:
        assert pb.bf16 and not pt.bf16
        rb = pb.unpack(ffx.ffx_expand(pb, to_dev(pack(pb, psis))))
        rt = pt.unpack(ffx.ffx_expand(pt, to_dev(pack(pt, psis))))
        assert pb.device_errors() == 0 and pt.device_errors() == 0
        worst = max(rel_l2(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(rb, rt))
        k = 5
        with ffx.PlanMany(specs[k:k + 1]) as one:
            r1 = ffx.ffx_expand(one, to_dev(psis[k].ravel())).cpu().numpy()
        assert np.array_equal(r1, rb[k].cpu().numpy().ravel())
    print(f"many bf16 vs tf32 phases: worst {worst:.2e}")
    assert worst < DENSITY_TOL


def test_many_tc_rejects_buffers_not_16_byte_aligned():
    """The tensor-core phases copy and store 16 bytes at a time: a buffer only
    8-byte aligned is refused on the host (FFX_EINVAL), before any launch."""
    ffx = require_gpu()
    specs = [((64, 32), (0.2, 0.2), 2.0, (3, 3)), ((32, 32, 32), (0.2,) * 3, 3.0, (2, 2, 2))]
    with ffx.PlanMany(specs, form="tc") as plan:
        assert plan.form == "tc"
        big = torch.zeros(plan.points + 1, dtype=torch.complex64, device="cuda")
        out = torch.empty(plan.points + 2, dtype=torch.float32, device="cuda")
        lib = ffx.load_library()
        rc = lib.ffx_expand(plan.handle, ctypes.c_void_p(big.data_ptr() + 8), 1,
                            ctypes.c_void_p(out.data_ptr()), None)
        assert rc == ffx.FFX_EINVAL
        rc = lib.ffx_expand(plan.handle, ctypes.c_void_p(big.data_ptr()), 1,
                            ctypes.c_void_p(out.data_ptr() + 8), None)
        assert rc == ffx.FFX_EINVAL
        assert plan.device_errors() == 0


def test_many_chain_new_buffers_modes_and_in_place_field():
    """Forward calls of a BF16 tensor-core plan run as chains whose first pass
    reads the call's input through tile maps made for that input buffer: a
    density call on a new buffer (maps remade) gives bitwise the same result,
    density and field calls alternate on different buffers, and a field call
    in place (1-D instance of 64 points, 2-D and 3-D instances) equals the
    out-of-place one and the FP64 oracle."""
    ffx = require_gpu()
    dims_set = [(64, 32, 48), (96, 32), (64,), (32, 128, 32)]
    specs, psis = mixed_specs(6, dims_override=dims_set)
    with ffx.PlanMany(specs, form="tc") as plan:
        assert plan.form == "tc" and plan.bf16
        x1 = to_dev(pack(plan, psis))
        x2 = x1.clone()
        r1 = ffx.ffx_expand(plan, x1).clone()
        f2 = ffx.ffx_expand_field(plan, x2).clone()
        r2 = ffx.ffx_expand(plan, x2)
        assert torch.equal(r1, r2)
        y = x1.clone()
        ffx.ffx_expand_field(plan, y, y)
        assert torch.equal(y, f2)
        assert plan.device_errors() == 0
        rho, field = r1.cpu().numpy(), f2.cpu().numpy()
        worst_d = worst_f = 0.0
        for (dims, dx, t, lam), p, off in zip(specs, psis, plan.offsets):
            ref = O.expand_field(p, dx, t, lam)
            m = p.size
            worst_d = max(worst_d, rel_l2(rho[off:off + m].reshape(dims), np.abs(ref) ** 2))
            worst_f = max(worst_f, rel_l2(field[off:off + m].reshape(dims), ref))
    print(f"many chain buffers/modes: worst density {worst_d:.2e}, worst field {worst_f:.2e}")
    assert worst_d < DENSITY_TOL and worst_f < FIELD_TOL


def test_many_backward_in_place_guard():
    """A backward call whose gradient buffer is its input: a 1-D instance of
    more than 64 points would read and write that buffer in one dense pass,
    so the call is refused (FFX_EUNSUPPORTED) on the host; without such an
    instance it runs and equals the out-of-place gradient."""
    ffx = require_gpu()
    rng = np.random.default_rng(21)
    with ffx.PlanMany([((96,), (0.1,), 1.0, (40,)), ((32, 32), (0.2, 0.2), 2.0, (30, 30))], form="tc") as plan:
        x = to_dev(rng.normal(size=plan.points).astype(np.complex64))
        g = to_dev(rng.normal(size=plan.points).astype(np.float32))
        with pytest.raises(ffx.FfxError) as ei:
            ffx.ffx_expand_backward(plan, x, g, x)
        assert ei.value.code == ffx.FFX_EUNSUPPORTED
    with ffx.PlanMany([((64,), (0.1,), 1.0, (40,)), ((32, 64), (0.2, 0.2), 2.0, (30, 30))], form="tc") as plan:
        x = to_dev((rng.normal(size=plan.points) + 1j * rng.normal(size=plan.points)).astype(np.complex64))
        g = to_dev(rng.normal(size=plan.points).astype(np.float32))
        ref = ffx.ffx_expand_backward(plan, x, g).clone()
        y = x.clone()
        ffx.ffx_expand_backward(plan, y, g, y)
        assert torch.equal(y, ref)
        assert plan.device_errors() == 0
