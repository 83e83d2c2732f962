"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  Together they are chosen so that a
plausible slip anywhere in the oracle (a dropped phase term, a wrong sign, a
wrong Nyquist/umklapp index, a transposed axis, a wrong normalisation) fails at
least one of them:

* closed forms: the free Gaussian packet (textbook), per axis and anisotropic
  in 3-D; the two-cloud interferometer formula printed in Sec. 6;
* the paper's exactness claim (Sec. 5.1, Sec. 7): its prescription eq. FF,
  written out term by term, equals the oracle, for even and odd M (umklapp),
  even and odd lam, 1-3 dimensions and non-integer offsets;
* brute force: split-step propagation on the vacuum-padded huge lattice
  (Sec. 2.3-2.4);
* special cases: t = 0 is exact subsampling; lam = 1 with abar = a is a
  unitary circulant; shifting abar by lam*dx shifts the output by one point;
* invariants: norm summed over the lam sub-lattice offsets (Parseval on the
  huge lattice), linearity; the ensemble mean of closed-form densities;
* limits: the far-field estimate eq. farfieldk is approached like 1/t;
* negative: the naive magnified DFT of Sec. 4.3 (eq. Psinaive) is wrong once
  the cloud outgrows the box;
* adjoint: dot-product identity and central finite differences.
"""

import json
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def grid(N, dx):
    return O.default_a(N, dx) + dx * np.arange(N)


def out_grid(N, dx, lam, a=None, abar=None):
    if a is None:
        a = O.default_a(N, dx)
    if abar is None:
        abar = O.default_abar(N, dx, lam, a)
    return abar + lam * dx * np.arange(N)


def gauss_t(x, t, sigma, c, k0):
    """Free Gaussian exp(-(x-c)^2/(2 sigma^2) + i k0 x) after time t (hbar=m=1)."""
    s2 = sigma ** 2 + 1j * t
    return np.sqrt(sigma ** 2 / s2) * np.exp(-(x - c - k0 * t) ** 2 / (2 * s2)
                                             + 1j * k0 * (x - 0.5 * k0 * t))


def gauss_periodic(x, t, sigma, c, k0, period):
    """The free Gaussian summed over its periodic images (the huge lattice is
    periodic with period lam*L); the images far away vanish to rounding."""
    return sum(gauss_t(x + m * period, t, sigma, c, k0) for m in range(-4, 5))


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,dx,lam,t,sigma,c,k0", [
    (256, 0.1, 16, 20.0, 1.0, 0.5, 2.0),
    (255, 0.1, 17, 12.0, 0.9, -0.7, -1.5),   # odd N, odd lam
    (200, 0.12, 10, 8.0, 1.2, 0.0, 3.0),
    (128, 0.1, 1, 2.0, 0.8, 0.3, 1.0),       # lam = 1: plain periodic propagation, wraps
])
def test_gaussian_closed_form_1d(N, dx, lam, t, sigma, c, k0):
    x = grid(N, dx)
    psi = gauss_t(x, 0.0, sigma, c, k0)
    out = O.expand_field(psi, (dx,), t, (lam,))
    ex = gauss_periodic(out_grid(N, dx, lam), t, sigma, c, k0, lam * N * dx)
    assert rel(out, ex) < 1e-11


def test_gaussian_closed_form_3d_anisotropic():
    """Different widths, momenta, spacings and lam on every axis: a transposed
    operand or an axis applied twice fails here."""
    dims, dx, lam = (80, 96, 72), (0.1, 0.09, 0.12), (6, 9, 4)
    t = 3.0
    sig, c, k0 = (0.5, 0.45, 0.55), (0.2, -0.1, 0.05), (1.0, -2.0, 0.5)
    axes_in = [grid(dims[j], dx[j]) for j in range(3)]
    psi = np.einsum("i,j,k->ijk", *[gauss_t(axes_in[j], 0, sig[j], c[j], k0[j]) for j in range(3)])
    out = O.expand_field(psi, dx, t, lam)
    ex = np.einsum("i,j,k->ijk", *[gauss_periodic(out_grid(dims[j], dx[j], lam[j]), t, sig[j], c[j],
                                                  k0[j], lam[j] * dims[j] * dx[j])
                                   for j in range(3)])
    assert rel(out, ex) < 1e-11


def test_two_cloud_interferometer_formula_and_fringe_readout():
    """Sec. 6: two Gaussians at y = -+D/2 (omega_perp = 1/sigma^2) evolve as
    psi(y,t) = (1 + i w t)^(-1/2) sum_+- A_+- exp[-w (2y -+ D)^2 / (8 (1 + i w t))].
    The fringe nearest y = 0 sits at y_peak = dtheta * t / D (eq. dphase2)."""
    N, dx, lam, t = 256, 0.05, 40, 6.0
    sigma, D = 0.5, 2.0
    w = 1.0 / sigma ** 2
    dtheta = 1.1
    Ap, Am = 1.0 * np.exp(1j * dtheta), 1.0     # + cloud leads by dtheta
    y = grid(N, dx)
    psi0 = Ap * np.exp(-w * (2 * y - D) ** 2 / 8) + Am * np.exp(-w * (2 * y + D) ** 2 / 8)
    out = O.expand_field(psi0, (dx,), t, (lam,))
    yb = out_grid(N, dx, lam)
    z = 1 + 1j * w * t
    ex = z ** -0.5 * (Ap * np.exp(-w * (2 * yb - D) ** 2 / (8 * z))
                      + Am * np.exp(-w * (2 * yb + D) ** 2 / (8 * z)))
    assert rel(out, ex) < 1e-11
    # fringe readout (eq. dphase2): clouds well separated (D = 10 sigma) so the
    # envelope's pull on the fringe, ~ 4 dtheta sigma^2 / D^2, stays < 0.05
    N2, dx2, lam2, t2 = 1024, 0.05, 2, 6.0
    sigma2, D2 = 0.3, 3.0
    w2 = 1.0 / sigma2 ** 2
    y2 = grid(N2, dx2)
    psi2 = Ap * np.exp(-w2 * (2 * y2 - D2) ** 2 / 8) + Am * np.exp(-w2 * (2 * y2 + D2) ** 2 / 8)
    rho = np.abs(O.expand_field(psi2, (dx2,), t2, (lam2,))) ** 2
    yb2 = out_grid(N2, dx2, lam2)
    est = float(O.fringe_phase(rho, yb2, D2, t2))
    assert abs(np.angle(np.exp(1j * (est - dtheta)))) < 0.1
    # the readout of the closed-form density (with its periodic images on the
    # lam N lattice) at the same points agrees
    z2 = 1 + 1j * w2 * t2
    period = lam2 * N2 * dx2
    ex2 = np.abs(sum(z2 ** -0.5 * (Ap * np.exp(-w2 * (2 * (yb2 + m * period) - D2) ** 2 / (8 * z2))
                                   + Am * np.exp(-w2 * (2 * (yb2 + m * period) + D2) ** 2 / (8 * z2)))
                     for m in range(-3, 4))) ** 2
    assert abs(float(O.fringe_phase(ex2, yb2, D2, t2)) - est) < 1e-8


# ---------------------------------------------------------------------------
# the paper's prescription and the brute force equal the definition
# ---------------------------------------------------------------------------

CASES_1D = [(16, 3, 2.0), (15, 4, 1.5), (15, 3, 0.7), (12, 2, 3.0), (9, 5, 0.3), (7, 6, 0.9),
            (32, 1, 0.5), (10, 8, 4.0)]


@pytest.mark.parametrize("N,lam,t", CASES_1D)
def test_recipe_equals_definition_1d(N, lam, t):
    rng = np.random.default_rng(N * 100 + lam)
    dx = 0.3
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)   # broadband: every bin matters
    d = O.expand_field(psi, (dx,), t, (lam,))
    r = O.recipe_field(psi, (dx,), t, (lam,))
    assert np.abs(d - r).max() < 1e-12 * np.abs(d).max()


def test_recipe_needs_umklapp_for_odd_M():
    """Leaving out the odd-M umklapp of Sec. 5.2 must break the equality, so
    the odd-M cases above really exercise it (a mistake planted in the
    oracle's recipe, on the CPU)."""
    N, lam, t, dx = 9, 4, 0.8, 0.3
    rng = np.random.default_rng(5)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    d = O.expand_field(psi, (dx,), t, (lam,))
    r = O.recipe_field(psi, (dx,), t, (lam,), umklapp=False)
    assert np.abs(d - r).max() > 1e-3 * np.abs(d).max()


@pytest.mark.parametrize("dims,lam,t", [((8, 9), (3, 2), 1.1), ((5, 6, 4), (2, 3, 2), 0.6),
                                        ((7, 4, 5), (3, 1, 2), 2.0)])
def test_recipe_equals_definition_nd(dims, lam, t):
    rng = np.random.default_rng(sum(dims))
    dx = tuple(0.2 + 0.05 * j for j in range(len(dims)))
    psi = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    d = O.expand_field(psi, dx, t, lam)
    r = O.recipe_field(psi, dx, t, lam)
    assert np.abs(d - r).max() < 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("frac", [0.3, 0.5, 0.77])
def test_recipe_equals_definition_noninteger_offset(frac):
    N, lam, dx, t = 16, 3, 0.3, 1.0
    a = O.default_a(N, dx)
    abar = a - (7 + frac) * dx
    rng = np.random.default_rng(11)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    d = O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    r = O.recipe_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    assert np.abs(d - r).max() < 1e-12 * np.abs(d).max()
    T = O.axis_matrix(N, dx, t, lam, a, abar)
    Td = O.axis_matrix_direct(N, dx, t, lam, a, abar)
    assert np.abs(T - Td).max() < 1e-13


@pytest.mark.parametrize("N,lam,t", CASES_1D)
def test_split_step_equals_definition(N, lam, t):
    rng = np.random.default_rng(N + 7 * lam)
    dx = 0.3
    psi = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    d = O.expand_field(psi, (dx,), t, (lam,))
    ss = O.split_step_axis(psi, dx, t, lam)
    assert np.abs(d - ss).max() < 1e-12 * np.abs(d).max()


def test_kernel_fft_step_matches_direct_sum():
    for N, lam, t in [(24, 5, 2.5), (17, 3, 0.4), (64, 2, 9.0)]:
        T = O.axis_matrix(N, 0.2, t, lam)
        Td = O.axis_matrix_direct(N, 0.2, t, lam)
        assert np.abs(T - Td).max() < 1e-13


# ---------------------------------------------------------------------------
# special cases and invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,lam,s", [(16, 3, -16), (15, 4, -22), (12, 2, 0), (10, 5, -13), (9, 1, 3)])
def test_t0_is_subsampling(N, lam, s):
    """At t = 0 the magnified lattice samples the vacuum-padded input:
    Psibar_nbar = psi_{(s + lam nbar) mod lam N} if that index is < N, else 0."""
    dx = 0.25
    a = O.default_a(N, dx)
    rng = np.random.default_rng(N)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    out = O.expand_field(psi, (dx,), 0.0, (lam,), a=(a,), abar=(a + s * dx,))
    idx = np.mod(s + lam * np.arange(N), lam * N)
    ex = np.where(idx < N, psi[np.minimum(idx, N - 1)], 0)
    assert np.abs(out - ex).max() < 1e-13


def test_lambda1_is_unitary_circulant():
    N, dx, t = 33, 0.2, 3.7
    T = O.axis_matrix(N, dx, t, 1, O.default_a(N, dx), O.default_a(N, dx))
    assert np.abs(T.conj().T @ T - np.eye(N)).max() < 1e-13
    assert np.abs(T - np.roll(np.roll(T, 1, 0), 1, 1)).max() < 1e-14


@pytest.mark.parametrize("N,lam", [(32, 4), (15, 3), (20, 5)])
def test_parseval_over_sublattice_offsets(N, lam):
    """The lam output lattices abar + r dx, r = 0..lam-1, tile the huge lattice;
    free flight there is unitary, so their summed norm equals the input norm."""
    dx, t = 0.2, 2.3
    a = O.default_a(N, dx)
    abar0 = O.default_abar(N, dx, lam, a)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    tot = sum(np.sum(np.abs(O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar0 + r * dx,))) ** 2)
              for r in range(lam))
    assert abs(tot - np.sum(np.abs(psi) ** 2)) < 1e-12 * np.sum(np.abs(psi) ** 2)


def test_output_offset_shift_moves_one_point():
    N, lam, dx, t = 24, 3, 0.2, 1.3
    a = O.default_a(N, dx)
    abar = O.default_abar(N, dx, lam, a)
    rng = np.random.default_rng(9)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    o1 = O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    o2 = O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar + lam * dx,))
    assert np.abs(o2[:-1] - o1[1:]).max() < 1e-13


def test_linearity_and_batch():
    dims, dx, lam, t = (6, 8, 10), (0.3, 0.25, 0.2), (2, 3, 4), 1.7
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2,) + dims) + 1j * rng.normal(size=(2,) + dims)
    f = O.expand_field(x, dx, t, lam)
    assert np.abs(f[0] - O.expand_field(x[0], dx, t, lam)).max() < 1e-13
    c = 0.3 - 1.2j
    g = O.expand_field(x[0] + c * x[1], dx, t, lam)
    assert np.abs(g - (f[0] + c * f[1])).max() < 1e-12


def test_ensemble_density_is_mean_of_closed_form_densities():
    """Ensembles of realizations (Sec. 1): the mean density over a batch of
    packets with different centres, widths, momenta and amplitudes equals the
    mean of their closed-form densities (free Gaussian, 2-D, separable).  A
    sum instead of a mean, a mean over a lattice axis, or a realization
    mixed into another fails here."""
    dims, dx, lam, t = (96, 80), (0.1, 0.12), (8, 5), 2.5
    params = [((0.6, 0.5), (0.3, -0.2), (1.5, 0.0), 1.0),
              ((0.45, 0.6), (-0.4, 0.1), (-1.0, 2.0), 0.5),
              ((0.55, 0.4), (0.0, 0.35), (0.5, -1.5), 2.0)]
    axes_in = [grid(dims[j], dx[j]) for j in range(2)]
    axes_out = [out_grid(dims[j], dx[j], lam[j]) for j in range(2)]
    psi = np.empty((len(params),) + dims, np.complex128)
    ex = np.zeros(dims)
    for r, (sig, c, k0, amp) in enumerate(params):
        psi[r] = amp * np.outer(*[gauss_t(axes_in[j], 0, sig[j], c[j], k0[j]) for j in range(2)])
        f = amp * np.outer(*[gauss_periodic(axes_out[j], t, sig[j], c[j], k0[j], lam[j] * dims[j] * dx[j])
                             for j in range(2)])
        ex += np.abs(f) ** 2 / len(params)
    got = O.ensemble_density(psi, dx, t, lam)
    assert got.shape == dims
    assert rel(got, ex) < 1e-10


# ---------------------------------------------------------------------------
# limits and negative tests
# ---------------------------------------------------------------------------

def test_far_field_limit_converges_like_inverse_t():
    """eq. farfieldk: t^d rho(xbar) -> |psi~(xbar/t)|^2.  For a generic
    (asymmetric, complex) state the leading correction is O(W^2/t)."""
    N, dx = 128, 0.1
    x = grid(N, dx)
    psi = np.exp(-x ** 2 / 2) * (1 + 0.6 * x) * np.exp(1j * x)
    errs = []
    for t in (25.0, 100.0, 400.0):
        lam = int(np.ceil((20 * t + N * dx) / (N * dx)))
        rho = O.expand_density(psi, (dx,), t, (lam,))
        ff = O.far_field_density(psi, (dx,), t, [out_grid(N, dx, lam)])
        errs.append(rel(rho, ff))
    assert errs[0] < 0.05
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.5 < e0 / e1 < 4.5


def _best_fit_rel(a, b):
    c = np.vdot(a, b) / np.vdot(a, a)
    return rel(c * a, b)


def test_naive_magnification_fails_when_cloud_outgrows_box():
    """Sec. 4.3 / FIG-3 setup: psi = exp(-x^2/2) cos(5x) on [-3, 3], M = 600.
    Once the cloud is wider than the box the naive eq. Psinaive scrambles the
    state; the oracle instead matches the closed form (a sum of two Gaussians
    moving at +-5)."""
    with open(os.path.join(HERE, "golden", "fig3_setup.json")) as fh:
        setup = json.load(fh)
    N = setup["M"]
    lo, hi = setup["x_range"]
    dx = (hi - lo) / N
    x = lo + dx * np.arange(N)
    k0 = setup["k0"]
    psi = np.exp(-x ** 2 / 2) * np.cos(k0 * x)
    t, lam = 1.0, 8
    a, abar = lo, lo - (lam - 1) * (hi - lo) / 2
    good = O.expand_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    xb = abar + lam * dx * np.arange(N)
    ex = 0.5 * (gauss_t(xb, t, 1.0, 0.0, k0) + gauss_t(xb, t, 1.0, 0.0, -k0))
    # the input box truncates the Gaussian at |x| = 3 (amplitude e^-4.5), so the
    # comparison is to that truncation level, not to rounding
    assert rel(good, ex) < 2e-2
    naive = O.naive_field(psi, (dx,), t, (lam,), a=(a,), abar=(abar,))
    assert _best_fit_rel(naive, ex) > 0.5


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

def test_adjoint_dot_product():
    dims, dx, lam, t = (6, 7, 10), (0.3, 0.25, 0.2), (2, 3, 5), 1.3
    rng = np.random.default_rng(4)
    x = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    y = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    lhs = np.vdot(O.expand_field(x, dx, t, lam), y)
    rhs = np.vdot(x, O.expand_adjoint(y, dx, t, lam))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_density_loss_gradient_finite_differences():
    dims, dx, lam, t = (6, 8, 5), (0.3, 0.25, 0.4), (3, 2, 4), 0.9
    rng = np.random.default_rng(8)
    psi = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    target = np.abs(O.expand_field(rng.normal(size=dims) + 0j, dx, t, lam)) ** 2

    def loss(p):
        return np.sum((O.expand_density(p, dx, t, lam) - target) ** 2)

    rho = O.expand_density(psi, dx, t, lam)
    g = O.density_loss_gradient(psi, 2 * (rho - target), dx, t, lam)
    for i in range(16):
        v = rng.normal(size=dims) + 1j * rng.normal(size=dims)
        eps = 1e-5 * np.linalg.norm(psi) / np.linalg.norm(v)
        fd = (loss(psi + eps * v) - loss(psi - eps * v)) / (2 * eps)
        an = np.real(np.vdot(g, v))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_sample_lines_matches_full():
    dims, dx, lam, t = (6, 7, 9), (0.3, 0.25, 0.2), (2, 3, 4), 1.1
    rng = np.random.default_rng(2)
    psi = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    full = O.expand_field(psi, dx, t, lam)
    assert np.abs(O.sample_lines(psi, dx, t, lam, 2, (4, 5)) - full[4, 5, :]).max() < 1e-13
    assert np.abs(O.sample_lines(psi, dx, t, lam, 0, (1, 8)) - full[:, 1, 8]).max() < 1e-13
    assert np.abs(O.sample_lines(psi, dx, t, lam, 1, (5, 0)) - full[5, :, 0]).max() < 1e-13


# ---------------------------------------------------------------------------
# detector readout (Sec. 6): column density and the fringe phase
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_column_density_of_separable_gaussian(axis):
    """A product of free Gaussians stays a product; integrating the density
    along one axis leaves the other two factors times that axis's sum of
    |G|^2 over the magnified points times their spacing lam dx (eq. wbx)."""
    dims, dx, lam, t = (64, 60, 72), (0.12, 0.13, 0.11), (3, 5, 2), 1.5
    sig, c, k0 = (0.5, 0.5, 0.45), (0.3, -0.2, 0.1), (0.5, -0.4, 0.7)
    axes_in = [grid(dims[j], dx[j]) for j in range(3)]
    psi = np.einsum("i,j,k->ijk", *[gauss_t(axes_in[j], 0, sig[j], c[j], k0[j]) for j in range(3)])
    col = O.column_density(psi[None], dx, t, lam, axis)[0]
    g = [np.abs(gauss_periodic(out_grid(dims[j], dx[j], lam[j]), t, sig[j], c[j], k0[j],
                               lam[j] * dims[j] * dx[j])) ** 2 for j in range(3)]
    other = [j for j in range(3) if j != axis]
    ex = np.outer(g[other[0]], g[other[1]]) * g[axis].sum() * lam[axis] * dx[axis]
    assert col.shape == (dims[other[0]], dims[other[1]])
    assert rel(col, ex) < 1e-9


def test_fringe_phase_vertex_and_nearest_peak():
    """The readout's own steps: on rho = exp(-(y - y*)^2 / w) the parabola
    through log rho is exact, so the vertex is y* to rounding; among several
    maxima the one nearest y = 0 is taken; a monotone row has none."""
    y = -3.0 + 0.1 * np.arange(61)
    D, t = 2.0, 5.0
    for ystar in (0.0, 0.037, -0.081, 0.2449):
        rho = np.exp(-(y - ystar) ** 2 / 0.3)
        assert abs(float(O.fringe_phase(rho, y, D, t)) - ystar * D / t) < 1e-12
    # fringes cos^2(pi (y - y0) / s) under a broad envelope: peaks at y0 + k s
    s_, y0 = 1.3, 0.41
    rho = np.exp(-y ** 2 / 50) * np.cos(np.pi * (y - y0) / s_) ** 2 + 1e-3
    est = float(O.fringe_phase(rho, y, D, t))
    assert abs(est * t / D - y0) < 0.02          # the k = 0 fringe, not k = -1 at y0 - s
    img = np.stack([rho, np.linspace(1, 2, 61)])  # second row: no interior maximum
    both = O.fringe_phase(img, y, D, t)
    assert both[0] == est and np.isnan(both[1])
    # the y axis may be any axis of the image
    assert O.fringe_phase(img.T, y, D, t, y_axis=0)[0] == est


# ---------------------------------------------------------------------------
# generalizations (Sec. 7): other spectra, positive-P pairs
# ---------------------------------------------------------------------------

def test_dispersion_free_particle_and_offsets():
    """omega = k^2/2 given as a table is the free map exactly; a constant
    offset omega + V only multiplies the field by exp(-i V t)."""
    dims, dx, lam, t = (24, 20), (0.3, 0.25), (3, 5), 2.5
    rng = np.random.default_rng(71)
    psi = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    ks = [O.fine_wavevectors(dims[j], dx[j], lam[j]) for j in range(2)]
    free = O.expand_field(psi, dx, t, lam)
    tab = O.expand_field(psi, dx, t, lam, omega=[0.5 * k * k for k in ks])
    assert np.abs(tab - free).max() < 1e-13 * np.abs(free).max()
    V = 0.37
    off = O.expand_field(psi, dx, t, lam, omega=[0.5 * ks[0] ** 2 + V, None])
    assert np.abs(off - np.exp(-1j * V * t) * free).max() < 1e-12 * np.abs(free).max()


@pytest.mark.parametrize("N,lam,m", [(16, 3, 5), (15, 4, -7), (12, 1, 3)])
def test_linear_dispersion_is_a_translation(N, lam, m):
    """omega = v k with v t = m dx moves the field by m huge-lattice points:
    Psibar_nbar = psi_n where s + lam nbar - n = m (mod lam N), vacuum
    elsewhere (eq. free0 with a linear spectrum)."""
    dx, t = 0.2, 1.7
    v = m * dx / t
    rng = np.random.default_rng(N + m)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    k = O.fine_wavevectors(N, dx, lam)
    out = O.expand_field(psi, (dx,), t, (lam,), omega=[v * k])
    a = O.default_a(N, dx)
    s0 = round((O.default_abar(N, dx, lam, a) - a) / dx)
    ex = np.zeros(N, complex)
    for nb in range(N):
        for n in range(N):
            if (s0 + lam * nb - n - m) % (lam * N) == 0:
                ex[nb] += psi[n]
    assert np.abs(out - ex).max() < 1e-12


def test_positive_p_pair():
    """psi+ = conj(psi) gives |Psibar|^2; the density is bilinear: it is
    linear in psi+ for fixed psi; and psi+ evolves by conj(T), so swapping
    the roles of the pair conjugates the product Psibar+ Psibar."""
    dims, dx, lam, t = (20, 18), (0.3, 0.25), (4, 3), 1.5
    rng = np.random.default_rng(5)
    psi = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    pp1 = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    pp2 = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    rho = O.positive_p_density(psi, np.conj(psi), dx, t, lam)
    assert np.abs(rho - O.expand_density(psi, dx, t, lam)).max() < 1e-12 * rho.max()
    lin = O.positive_p_density(psi, pp1 + 2.5 * pp2, dx, t, lam)
    assert np.abs(lin - O.positive_p_density(psi, pp1, dx, t, lam)
                  - 2.5 * O.positive_p_density(psi, pp2, dx, t, lam)).max() < 1e-11 * np.abs(lin).max()
    # Re(conj(T) a * T b) = Re(T conj(a) * conj(T) conj(b)): the pair (conj a, conj b) swapped
    r1 = O.positive_p_density(psi, pp1, dx, t, lam)
    r2 = O.positive_p_density(np.conj(pp1), np.conj(psi), dx, t, lam)
    assert np.abs(r1 - r2).max() < 1e-12 * np.abs(r1).max()
    # and it is not |.|^2 of either field alone
    assert np.abs(r1 - O.expand_density(psi, dx, t, lam)).max() > 1e-3
