"""Sec. 7 generalizations on the GPU: other spectra (a separable dispersion
replacing k^2/2) and positive-P pairs, against the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
from gpu_common import DENSITY_TOL, FIELD_TOL, random_field, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffx():
    return require_gpu()


def spectra(dims, dx, lam, kind):
    ks = [O.fine_wavevectors(dims[j], dx[j], lam[j]) for j in range(len(dims))]
    if kind == "quartic":      # a stiffened spectrum: k^2/2 + 0.02 k^4
        return [0.5 * k * k + 0.02 * k ** 4 for k in ks]
    if kind == "masses":       # anisotropic masses, free on the last axis
        return [k * k / (2 * m) for k, m in zip(ks[:-1], (0.7, 1.9))] + [None]
    if kind == "relativistic":  # sqrt(k^2 + 1), a massive relativistic branch
        return [np.sqrt(k * k + 1.0) for k in ks]
    raise ValueError(kind)


@pytest.mark.parametrize("form,fused", [("auto", True), ("dense", False), ("fold", False), ("paper", False),
                                        ("tc", False)])
@pytest.mark.parametrize("kind", ["quartic", "masses", "relativistic"])
def test_dispersion_matches_oracle(ffx, form, fused, kind):
    dims, dx, lam, t = (64, 48, 64), (0.25, 0.3, 0.2), (5, 7, 3), 2.0
    rng = np.random.default_rng(len(kind) * 13 + len(form))
    psi = random_field(rng, (2,) + dims)
    omega = spectra(dims, dx, lam, kind)
    ref = O.expand_field(psi, dx, t, lam, omega=omega)
    with ffx.Plan(dims, dx, t, lam, form=form, fused=fused, omega=omega) as plan:
        field = ffx.ffx_expand_field(plan, to_dev(psi)).cpu().numpy()
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        assert plan.device_errors() == 0
    ef, ed = rel_l2(field, ref), rel_l2(rho, np.abs(ref) ** 2)
    print(f"dispersion {kind} {form}: field {ef:.2e} density {ed:.2e}")
    assert ef < FIELD_TOL and ed < DENSITY_TOL


def test_linear_dispersion_translates(ffx):
    """omega = v k with v t = m dx: the field moves by m huge-lattice points."""
    N, dx, lam, t, m = 64, 0.2, 3, 1.7, 9
    v = m * dx / t
    rng = np.random.default_rng(3)
    psi = random_field(rng, (1, N))
    with ffx.Plan((N,), (dx,), t, (lam,), omega=[v * O.fine_wavevectors(N, dx, lam)]) as plan:
        out = ffx.ffx_expand_field(plan, to_dev(psi)).cpu().numpy()[0]
    a = O.default_a(N, dx)
    s0 = round((O.default_abar(N, dx, lam, a) - a) / dx)
    ex = np.zeros(N, complex)
    for nb in range(N):
        for n in range(N):
            if (s0 + lam * nb - n - m) % (lam * N) == 0:
                ex[nb] += psi[0, n]
    assert np.abs(out - ex).max() < 1e-5 * np.abs(psi).max()


@pytest.mark.parametrize("fused,accumulate", [(True, False), (False, False), (True, True), (False, True)])
def test_positive_p_pairs(ffx, fused, accumulate):
    dims, dx, lam, t = (64, 32, 48), (0.25, 0.25, 0.3), (9, 4, 6), 3.0
    rng = np.random.default_rng(11)
    batch = 2
    psi = random_field(rng, (batch,) + dims)
    psp = random_field(rng, (batch,) + dims)
    ref = O.positive_p_density(psi, psp, dx, t, lam)
    with ffx.Plan(dims, dx, t, lam, fused=fused, accumulate=accumulate) as plan:
        got = ffx.ffx_expand_positive_p(plan, to_dev(psi), to_dev(psp)).cpu().numpy()
        classical = ffx.ffx_expand_positive_p(plan, to_dev(psi), to_dev(np.conj(psi))).cpu().numpy()
        assert plan.device_errors() == 0
    if accumulate:
        ref = ref.sum(0)
    e = rel_l2(got, ref)
    ec = rel_l2(classical, (np.abs(O.expand_field(psi, dx, t, lam)) ** 2).sum(0) if accumulate
                else np.abs(O.expand_field(psi, dx, t, lam)) ** 2)
    print(f"positive-P fused={fused} acc={accumulate}: {e:.2e}, classical limit {ec:.2e}")
    assert e < DENSITY_TOL and ec < DENSITY_TOL


@pytest.mark.parametrize("kind", ["quartic", "masses"])
def test_dispersion_and_positive_p_on_the_bf16_chain(ffx, kind):
    """Every axis on the BF16 tensor-core kernel (96 and 128 points): the
    forward calls run as a BF16 chain (input split, passes from the last axis
    to the first, planes between them) with the dispersion tables and for
    both fields of a positive-P pair."""
    dims, dx, lam, t = (128, 96, 128), (0.25, 0.3, 0.2), (5, 7, 3), 2.0
    batch = 2
    rng = np.random.default_rng(len(kind) + 400)
    psi = random_field(rng, (batch,) + dims)
    psp = random_field(rng, (batch,) + dims)
    omega = spectra(dims, dx, lam, kind)
    ref = O.expand_field(psi, dx, t, lam, omega=omega)
    with ffx.Plan(dims, dx, t, lam, form="tc", bf16=True, omega=omega) as plan:
        assert plan.bf16_chain(batch)
        field = ffx.ffx_expand_field(plan, to_dev(psi)).cpu().numpy()
        rho = ffx.ffx_expand(plan, to_dev(psi)).cpu().numpy()
        pp = ffx.ffx_expand_positive_p(plan, to_dev(psi), to_dev(psp)).cpu().numpy()
        assert plan.device_errors() == 0
    refp = O.positive_p_density(psi, psp, dx, t, lam, omega=omega)
    ef, ed, ep = rel_l2(field, ref), rel_l2(rho, np.abs(ref) ** 2), rel_l2(pp, refp)
    print(f"bf16 chain, dispersion {kind}: field {ef:.2e} density {ed:.2e} positive-P {ep:.2e}")
    assert ef < FIELD_TOL and ed < DENSITY_TOL and ep < DENSITY_TOL
