"""The failure path of the bounded device waits (FFX_ETIMEOUT).

The fused one-launch path of a small lattice has blocks that wait for other
blocks: a grid-wide barrier between its passes and per-tile counters.  With a
poll budget of one, the first blocks to arrive give up on those waits at once.
Nothing faults or hangs: such a block stops its passes, drains its own bulk
copies and tensor-core work with the normal bound, frees its tensor memory and
counts the timeout.  The test checks that the launch returns, that the count
is positive, that the next call on the plan reports FFX_ETIMEOUT without
launching, and that the plan (budget restored) and a fresh plan in the same
process still match the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import DENSITY_TOL, rel_l2, require_gpu, to_dev
from paper_1602_03395_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["auto", "dense"])
def test_cross_block_wait_runs_out_and_reports(form):
    ffx = require_gpu()
    w = inputs.config_two_cloud()
    psi = w.batch_array(1)
    ref = np.abs(O.expand_field(psi, w.dx, w.t, w.lam)) ** 2
    x = to_dev(psi)
    plan = ffx.Plan(w.dims, w.dx, w.t, w.lam, form=form)
    try:
        assert plan.fused and plan.fused_max_batch >= 1
        assert plan.launches_per_call(batch=1) == 1
        good = ffx.ffx_expand(plan, x).cpu().numpy()
        assert plan.device_errors() == 0
        plan.set_wait_limit(1)
        ffx.ffx_expand(plan, x)           # the launch gives up on its waits and returns
        torch.cuda.synchronize()
        n = plan.device_errors()
        print(f"{form}: timeouts counted {n}")
        assert n > 0
        with pytest.raises(ffx.FfxError) as ei:
            ffx.ffx_expand(plan, x)       # reports the earlier timeout, launches nothing
        assert ei.value.code == ffx.FFX_ETIMEOUT
        plan.set_wait_limit(0)
        again = ffx.ffx_expand(plan, x).cpu().numpy()
        assert plan.device_errors() == n  # no new timeout
        assert np.array_equal(again, good)
        assert rel_l2(again, ref) < DENSITY_TOL
    finally:
        plan.close()
    with ffx.Plan(w.dims, w.dx, w.t, w.lam, form=form) as fresh:
        e = rel_l2(ffx.ffx_expand(fresh, x).cpu().numpy(), ref)
        assert fresh.device_errors() == 0
    assert e < DENSITY_TOL


def test_wait_limit_argument_checks():
    ffx = require_gpu()
    with ffx.Plan((32, 32), (0.25, 0.25), 1.0, (3, 3)) as plan:
        with pytest.raises(ffx.FfxError) as ei:
            plan.set_wait_limit(-1)
        assert ei.value.code == ffx.FFX_EINVAL
        plan.set_wait_limit(0)
