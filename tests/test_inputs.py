"""Seeded input generators: deterministic, right shapes, complex64."""

import numpy as np

from paper_1602_03395_gb300 import inputs


def test_workloads_deterministic_and_typed():
    for w in [inputs.config_1d(), inputs.config_two_cloud(), inputs.config_quasicondensate(batch=2)]:
        a = w.realization(0)
        b = w.realization(0)
        c = w.realization(1)
        assert a.dtype == np.complex64 and a.shape == tuple(w.dims)
        assert np.array_equal(a, b)
        assert not np.array_equal(a, c) or w.batch == 1
        assert np.isfinite(a).all()


def test_shapes_match_workloads():
    w = inputs.config_1d()
    psi = w.realization(0)
    x = inputs.axis_coords(512, 0.1)
    assert abs(psi).max() <= 1.0 + 1e-6
    assert abs(psi[np.abs(x) > 20]).max() == 0.0  # Thomas-Fermi support
    q = inputs.config_quasicondensate(batch=1).realization(0)
    assert abs(q[0, 0, :]).max() == 0.0           # outside the transverse TF radius
    assert np.allclose(np.abs(q[16, 16, 256]), 1.0, atol=1e-3) or np.abs(q[16, 16, 256]) < 1.0


def test_mixed_batch_draws():
    ws = inputs.config_mixed_batch(count=50)
    assert {tuple(w.dims) for w in ws} <= set(inputs.MIXED_SHAPES)
    lams = [w.lam[0] for w in ws]
    assert min(lams) >= 10 and max(lams) <= 100
    assert all(w.t == 4.0 * w.lam[0] for w in ws)
