"""FP64 CPU oracle for the free-flight expansion onto a magnified lattice.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant with the CUDA path.

What it computes (Deuar, arXiv:1602.03395, Sec. 5.1, eqs. ex1, time, ex4 sampled
at wbx).  The initial field psi_n lives on the lattice x_n = a + n dx
(eq. xj), n = 0..N-1, and is surrounded by vacuum (eq. vacuum).  Free flight
for a time t is carried out exactly on the periodic "huge" lattice of lam*N
points with the same spacing dx, whose wavevectors are the fine set
k_u = 2 pi l(u) / (lam L), l(u) the symmetric index of eq. kj on lam*N points
(eq. ulk).  The result is sampled on the magnified lattice
xbar_nbar = abar + nbar * lam * dx (eq. wbx).  In one dimension this is the
linear map

    Psibar_nbar = sum_n T[nbar, n] psi_n,
    T[nbar, n]  = (1/(lam N)) sum_u exp(i k_u (xbar_nbar - x_n) - i t k_u^2 / 2),

with hbar = m = 1 (any physical hbar t / m goes into t).  Every phase of the
map is exp(i sum_j ...), so the d-dimensional map is the tensor product of
the 1-D maps of each axis; the oracle applies T_j along axis j with a BLAS
matrix product.  The paper's prescription (eq. FF) reaches this map exactly
(Sec. 5.1 derivation; Sec. 7 conclusion), so the definition, not the
recipe, is what the oracle evaluates.

``recipe_field`` below additionally writes out the paper's prescription
(eqs. FFpsi, presf, presB, presA, FFaux, with the odd-M umklapp of Sec. 5.2)
in its own, non-separable form.  It is used only by the oracle's own tests,
to show that the recipe and the definition agree.

Readings of points the paper leaves open are listed in the module-level
docstrings of the functions that take them.  Parity of every function is
pinned by ``tests/test_oracle_pins.py``.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "symmetric_index",
    "default_a",
    "default_abar",
    "axis_matrix",
    "axis_matrix_direct",
    "expand_field",
    "expand_density",
    "ensemble_density",
    "expand_adjoint",
    "density_loss_gradient",
    "split_step_axis",
    "recipe_field",
    "naive_field",
    "far_field_density",
    "sample_lines",
    "column_density",
    "fringe_phase",
    "fine_wavevectors",
    "positive_p_density",
]


# ---------------------------------------------------------------------------
# lattice conventions
# ---------------------------------------------------------------------------

def symmetric_index(M: int) -> np.ndarray:
    """Integer wavevector multipliers l(m), m = 0..M-1, of eq. kj.

    l = m for m < M/2 and l = m - M otherwise.  For even M the Nyquist bin
    m = M/2 maps to l = -M/2 (the paper's piecewise rule, Sec. 2.3).
    """
    m = np.arange(M, dtype=np.int64)
    return np.where(2 * m < M, m, m - M)


def default_a(N: int, dx: float) -> float:
    """Input offset a = -L/2: the input box is centred on x = 0.

    The workloads do not state a; the paper centres its huge lattice the same
    way (Sec. 3, abar = -L/2 for the 1-D brute-force run)."""
    return -0.5 * N * dx


def default_abar(N: int, dx: float, lam: int, a: float) -> float:
    """Output offset abar = a + s dx with s = -floor((lam-1) N / 2).

    This centres the magnified box on the input box (abar = a - (lam-1) L / 2)
    whenever (lam-1) N is even, and keeps s an integer otherwise."""
    s = -(((lam - 1) * N) // 2)
    return a + s * dx


# ---------------------------------------------------------------------------
# the definition: free flight on the vacuum-padded huge lattice
# ---------------------------------------------------------------------------

def _fine_wavevectors(N: int, dx: float, lam: int) -> np.ndarray:
    """k_u = 2 pi l(u) / (lam L), u = 0..lam N - 1 (eq. ulk, huge lattice)."""
    L = N * dx
    return 2.0 * np.pi * symmetric_index(lam * N).astype(np.float64) / (lam * L)


def fine_wavevectors(N: int, dx: float, lam: int) -> np.ndarray:
    """The lam N huge-lattice wavevectors k_u in index order u (eq. ulk): the
    points at which a dispersion omega is sampled for ``omega=`` below."""
    return _fine_wavevectors(N, dx, lam)


def axis_matrix(N: int, dx: float, t: float, lam: int,
                a: float | None = None, abar: float | None = None, omega=None) -> np.ndarray:
    """Dense 1-D free-flight map T[nbar, n] (complex128, N x N).

    T[nbar, n] = (1/(lam N)) sum_u exp(i k_u (xbar_nbar - x_n) - i t k_u^2/2).

    Other spectra (Sec. 7, Generalizations): with ``omega`` (lam N values,
    omega[u] at k_u) the free-particle phase t k_u^2 / 2 becomes t omega[u]
    (the momentum-space evolution exp(-i t omega_k) replaces eq. free0).

    Writing s = (abar - a)/dx = s0 + sf (s0 integer, 0 <= sf < 1) gives
    xbar_nbar - x_n = (s0 + lam nbar - n + sf) dx, and since
    k_u * m * dx = 2 pi l(u) m / (lam N) for integer m, T is a lookup
    T[nbar, n] = K[(s0 + lam nbar - n) mod lam N] into the huge-lattice
    propagator K[m] = (1/(lam N)) sum_u exp(2 pi i u m/(lam N))
    * exp(i k_u sf dx - i t k_u^2 / 2), evaluated with one inverse FFT of
    length lam N (a library step).  ``axis_matrix_direct`` sums the same
    definition term by term for small sizes.
    """
    lam = int(lam)
    if lam < 1 or N < 1:
        raise ValueError("need lam >= 1 and N >= 1")
    if a is None:
        a = default_a(N, dx)
    if abar is None:
        abar = default_abar(N, dx, lam, a)
    NN = lam * N
    k = _fine_wavevectors(N, dx, lam)
    s = (abar - a) / dx
    s0 = math.floor(s)
    sf = s - s0
    if omega is None:
        phase = 0.5 * t * k * k
    else:
        omega = np.asarray(omega, dtype=np.float64)
        if omega.shape != (NN,):
            raise ValueError("omega must hold lam*N values")
        phase = t * omega
    spec = np.exp(-1j * phase + 1j * k * (sf * dx))
    K = np.fft.ifft(spec)  # includes the 1/(lam N)
    nbar = np.arange(N, dtype=np.int64)
    n = np.arange(N, dtype=np.int64)
    idx = np.mod(s0 + lam * nbar[:, None] - n[None, :], NN)
    return K[idx]


def axis_matrix_direct(N: int, dx: float, t: float, lam: int,
                       a: float | None = None, abar: float | None = None) -> np.ndarray:
    """The same T, summed literally over the lam*N fine wavevectors (small N only)."""
    lam = int(lam)
    if a is None:
        a = default_a(N, dx)
    if abar is None:
        abar = default_abar(N, dx, lam, a)
    k = _fine_wavevectors(N, dx, lam)
    xbar = abar + np.arange(N) * lam * dx
    x = a + np.arange(N) * dx
    delta = xbar[:, None] - x[None, :]
    ph = np.exp(1j * delta[:, :, None] * k[None, None, :] - 0.5j * t * k * k)
    return ph.sum(axis=2) / (lam * N)


def _as_tuple(v, d, name):
    if np.isscalar(v):
        return (v,) * d
    v = tuple(v)
    if len(v) != d:
        raise ValueError(f"{name} must have {d} entries")
    return v


def _axis_matrices(dims, dx, t, lam, a, abar, omega=None):
    d = len(dims)
    dx = _as_tuple(dx, d, "dx")
    lam = _as_tuple(lam, d, "lam")
    a = _as_tuple(a, d, "a") if a is not None else (None,) * d
    abar = _as_tuple(abar, d, "abar") if abar is not None else (None,) * d
    omega = tuple(omega) if omega is not None else (None,) * d
    if len(omega) != d:
        raise ValueError(f"omega must have {d} entries")
    return [axis_matrix(int(dims[j]), float(dx[j]), float(t), int(lam[j]), a[j], abar[j], omega[j])
            for j in range(d)]


def _apply_along(T: np.ndarray, psi: np.ndarray, axis: int) -> np.ndarray:
    out = np.tensordot(T, psi, axes=([1], [axis]))  # new axis in front
    return np.moveaxis(out, 0, axis)


def expand_field(psi0, dx, t, lam, a=None, abar=None, omega=None) -> np.ndarray:
    """Psibar on the magnified lattice for a batch psi0[..., M_1, ..., M_d].

    ``dx``, ``lam``, ``a``, ``abar`` are scalars or per-axis sequences; the last
    len(dx) axes (or 1 if scalar) are the lattice axes.  psi0 is promoted to
    complex128 first, so an input already rounded to complex64 is taken as
    exact.  ``omega``: per axis None (free particle) or the lam_j N_j values of
    a separable dispersion omega_j at ``fine_wavevectors`` (Sec. 7).
    """
    psi = np.asarray(psi0).astype(np.complex128)
    d = len(dx) if not np.isscalar(dx) else 1
    dims = psi.shape[psi.ndim - d:]
    Ts = _axis_matrices(dims, dx, t, lam, a, abar, omega)
    for j in range(d):
        psi = _apply_along(Ts[j], psi, psi.ndim - d + j)
    return psi


def expand_density(psi0, dx, t, lam, a=None, abar=None, omega=None) -> np.ndarray:
    """rho = |Psibar|^2 per realization (Sec. 2, the measured density)."""
    f = expand_field(psi0, dx, t, lam, a, abar, omega)
    return f.real ** 2 + f.imag ** 2


def ensemble_density(psi0, dx, t, lam, a=None, abar=None) -> np.ndarray:
    """Mean density over the leading (realization) axis of psi0."""
    return expand_density(psi0, dx, t, lam, a, abar).mean(axis=0)


def expand_adjoint(g, dx, t, lam, a=None, abar=None) -> np.ndarray:
    """Apply the adjoint map T^H = T_1^H x ... x T_d^H to g[..., M_1..M_d]."""
    g = np.asarray(g).astype(np.complex128)
    d = len(dx) if not np.isscalar(dx) else 1
    dims = g.shape[g.ndim - d:]
    Ts = _axis_matrices(dims, dx, t, lam, a, abar)
    for j in range(d):
        g = _apply_along(Ts[j].conj().T, g, g.ndim - d + j)
    return g


def density_loss_gradient(psi0, grad_rho, dx, t, lam, a=None, abar=None) -> np.ndarray:
    """Gradient of a real loss of rho = |T psi0|^2 with respect to psi0.

    With dL/drho = grad_rho given, the gradient in the convention
    dL/dRe(psi0) + i dL/dIm(psi0) is T^H (2 grad_rho * T psi0).
    """
    field = expand_field(psi0, dx, t, lam, a, abar)
    return expand_adjoint(2.0 * np.asarray(grad_rho, dtype=np.float64) * field,
                          dx, t, lam, a, abar)


def sample_lines(psi0, dx, t, lam, axis: int, index: tuple, a=None, abar=None) -> np.ndarray:
    """One output line of Psibar along lattice axis ``axis`` (single realization).

    ``index`` gives the output indices nbar_j of every other lattice axis, in
    order.  Uses the separable form: contract the other axes with the rows of
    their T_j first (cost ~ M per line), then apply T_axis.  Lets large
    outputs be checked line by line.
    """
    psi = np.asarray(psi0).astype(np.complex128)
    d = psi.ndim
    Ts = _axis_matrices(psi.shape, dx, t, lam, a, abar)
    other = [j for j in range(d) if j != axis]
    if len(index) != len(other):
        raise ValueError("index must name one output index per other axis")
    v = psi
    # contract other axes from the last to the first so positions stay valid
    for j, nb in sorted(zip(other, index), reverse=True):
        v = np.tensordot(v, Ts[j][nb], axes=([j], [0]))
    return Ts[axis] @ v


def positive_p_density(psi0, psi0_plus, dx, t, lam, a=None, abar=None, omega=None) -> np.ndarray:
    """Density of a positive-P pair after free flight (Sec. 7, Generalizations).

    The two independent fields psi (for the annihilation field) and psi+ (for
    the creation field) evolve by the map and by its complex conjugate:
    Psibar = T psi0, Psibar+ = conj(T) psi0+ (the conjugate equation of
    motion; T the per-axis maps as in ``expand_field``).  The normally
    ordered density is Re(Psibar+ Psibar).  With psi0+ = conj(psi0) it is
    |Psibar|^2.
    """
    psi = np.asarray(psi0).astype(np.complex128)
    psp = np.asarray(psi0_plus).astype(np.complex128)
    if psi.shape != psp.shape:
        raise ValueError("psi0 and psi0_plus must have the same shape")
    d = len(dx) if not np.isscalar(dx) else 1
    dims = psi.shape[psi.ndim - d:]
    Ts = _axis_matrices(dims, dx, t, lam, a, abar, omega)
    for j in range(d):
        psi = _apply_along(Ts[j], psi, psi.ndim - d + j)
        psp = _apply_along(Ts[j].conj(), psp, psp.ndim - d + j)
    return (psp * psi).real


# ---------------------------------------------------------------------------
# detector readout (Sec. 6)
# ---------------------------------------------------------------------------

def column_density(psi0, dx, t, lam, axis: int, a=None, abar=None) -> np.ndarray:
    """The detector image: the density integrated along lattice axis ``axis``.

    Sec. 6 takes the image at the detector as the density integrated over the
    imaging direction, rho(x, y) = integral dz |Psi|^2 (Fig. 4).  On the
    magnified lattice the points along that axis are lam_axis dx_axis apart
    (eq. wbx), so the integral is the sum of |Psibar|^2 over the axis times
    lam_axis dx_axis.  ``axis`` counts lattice axes (0 .. d-1); the result keeps
    the batch axes and drops that one.
    """
    rho = expand_density(psi0, dx, t, lam, a, abar)
    d = len(dx) if not np.isscalar(dx) else 1
    dxs = _as_tuple(dx, d, "dx")
    lams = _as_tuple(lam, d, "lam")
    if not 0 <= axis < d:
        raise ValueError("axis out of range")
    return rho.sum(axis=rho.ndim - d + axis) * (lams[axis] * dxs[axis])


def fringe_phase(image, ybar, D: float, t: float, y_axis: int = -1) -> np.ndarray:
    """Relative phase of two clouds split by D along y, read from the fringes
    (eq. dphase2, hbar = m = 1): Delta theta_0 = y_peak D / t, where y_peak is
    the position of the density peak nearest y = 0.

    ``image`` is a density (or detector image) sampled at positions ``ybar``
    (equally spaced) along ``y_axis``; every position along its other axes
    gives one estimate.  The peak is the interior local maximum
    (rho[j] > rho[j-1] and rho[j] >= rho[j+1], compared in the image's own
    precision) with the smallest |ybar[j]|, the lower j on a tie; its position
    is refined to the vertex of the parabola through log rho at j-1, j, j+1
    (in FP64; no refinement when a value is not positive or the parabola is
    flat).  A row without an interior maximum gives NaN.  Phases are not
    wrapped.
    """
    img = np.moveaxis(np.asarray(image), y_axis, -1)
    y = np.asarray(ybar, dtype=np.float64)
    ny = img.shape[-1]
    if y.shape != (ny,):
        raise ValueError("ybar must give one position per image point along y")
    dy = (y[-1] - y[0]) / (ny - 1) if ny > 1 else 0.0
    flat = img.reshape(-1, ny)
    out = np.full(flat.shape[0], np.nan)
    for r, row in enumerate(flat):
        best = -1
        for j in range(1, ny - 1):
            if row[j] > row[j - 1] and row[j] >= row[j + 1]:
                if best < 0 or abs(y[j]) < abs(y[best]):
                    best = j
        if best < 0:
            continue
        rm, r0, rp = (float(v) for v in row[best - 1:best + 2])
        shift = 0.0
        if rm > 0 and r0 > 0 and rp > 0:
            lm, l0, lp = math.log(rm), math.log(r0), math.log(rp)
            curv = lm - 2.0 * l0 + lp
            if curv != 0.0:
                shift = 0.5 * (lm - lp) / curv
        out[r] = (y[best] + shift * dy) * D / t
    return out.reshape(img.shape[:-1])


# ---------------------------------------------------------------------------
# second, independent route: brute-force split step on the huge lattice
# ---------------------------------------------------------------------------

def split_step_axis(psi: np.ndarray, dx: float, t: float, lam: int,
                    a: float | None = None, abar: float | None = None) -> np.ndarray:
    """Brute force along the last axis: pad with vacuum to lam*N points,
    transform, apply the free-flight phase, transform back, and take every
    lam-th point starting at offset s (Sec. 2.3 eqs. Psiwtm, free0, Psin on
    the huge lattice).  Requires an integer s = (abar - a)/dx."""
    psi = np.asarray(psi).astype(np.complex128)
    N = psi.shape[-1]
    lam = int(lam)
    if a is None:
        a = default_a(N, dx)
    if abar is None:
        abar = default_abar(N, dx, lam, a)
    s = (abar - a) / dx
    if abs(s - round(s)) > 1e-9:
        raise ValueError("split_step_axis needs abar - a to be a multiple of dx")
    s = int(round(s))
    NN = lam * N
    pad = np.zeros(psi.shape[:-1] + (NN,), np.complex128)
    pad[..., :N] = psi  # the huge lattice starts at x = a
    k = _fine_wavevectors(N, dx, lam)
    out = np.fft.ifft(np.fft.fft(pad, axis=-1) * np.exp(-0.5j * t * k * k), axis=-1)
    return out[..., np.mod(s + lam * np.arange(N), NN)]


# ---------------------------------------------------------------------------
# the paper's prescription written out as printed (tests of the oracle only)
# ---------------------------------------------------------------------------

def recipe_field(psi0: np.ndarray, dx, t: float, lam, a=None, abar=None,
                 umklapp: bool = True) -> np.ndarray:
    """Eq. FF evaluated in its own non-separable form, one term per q-tuple.

    For every q = (q_1..q_d), q_j in [0, lam_j):
      alpha_j = q_j dk_j / lam_j,
      A = FFT[psi * exp(-i alpha.(x - a))]                              (presA)
      B = IFFT[A * exp(i k.(abar - a - (k + 2 alpha) t / 2))]          (presB)
          with k_j(m) -> -dk_j (M_j + 1)/2 at m = (M_j - 1)/2 when M_j is
          odd and q_j >= lam_j / 2 (odd-M umklapp, Sec. 5.2)
      f = (1/lam) exp(i alpha.(xbar - a - alpha t / 2))                 (presf)
      Psibar[nbar] += f[nbar] * B[n''], n''_j = (nbar_j lam_j) mod M_j  (FFpsi, FFaux)
    IFFT carries the 1/M of eq. iDFT.  Cost prod(lam) * M log M: tiny inputs.
    ``umklapp=False`` leaves the odd-M correction out; it exists so a test can
    show that the correction is needed.
    """
    psi = np.asarray(psi0).astype(np.complex128)
    dims = psi.shape
    d = len(dims)
    dx = _as_tuple(dx, d, "dx")
    lam = tuple(int(v) for v in _as_tuple(lam, d, "lam"))
    a = _as_tuple(a, d, "a") if a is not None else tuple(default_a(dims[j], dx[j]) for j in range(d))
    if abar is None:
        abar = tuple(default_abar(dims[j], dx[j], lam[j], a[j]) for j in range(d))
    else:
        abar = _as_tuple(abar, d, "abar")
    L = [dims[j] * dx[j] for j in range(d)]
    dk = [2 * np.pi / L[j] for j in range(d)]
    lam_tot = int(np.prod(lam))
    # per-axis grids, broadcast to d dimensions
    def bshape(j):
        s = [1] * d
        s[j] = dims[j]
        return s
    xa = [(np.arange(dims[j]) * dx[j]).reshape(bshape(j)) for j in range(d)]        # x - a
    xbar_a = [(abar[j] - a[j] + np.arange(dims[j]) * lam[j] * dx[j]).reshape(bshape(j))
              for j in range(d)]                                                   # xbar - a
    nii = [np.mod(np.arange(dims[j]) * lam[j], dims[j]) for j in range(d)]
    out = np.zeros(dims, np.complex128)
    for q in itertools.product(*[range(l) for l in lam]):
        alpha = [q[j] * dk[j] / lam[j] for j in range(d)]
        pre = np.ones(dims, np.complex128)
        for j in range(d):
            pre = pre * np.exp(-1j * alpha[j] * xa[j])
        A = np.fft.fftn(psi * pre)
        ph = np.zeros(dims, np.float64)
        for j in range(d):
            kj = dk[j] * symmetric_index(dims[j]).astype(np.float64)
            if umklapp and dims[j] % 2 == 1 and 2 * q[j] >= lam[j]:
                kj[(dims[j] - 1) // 2] = -dk[j] * (dims[j] + 1) / 2
            kj = kj.reshape(bshape(j))
            ph = ph + kj * (abar[j] - a[j] - (kj + 2 * alpha[j]) * t / 2)
        B = np.fft.ifftn(A * np.exp(1j * ph))
        f = np.full(dims, 1.0 / lam_tot, np.complex128)
        for j in range(d):
            f = f * np.exp(1j * alpha[j] * (xbar_a[j] - alpha[j] * t / 2))
        out += f * B[np.ix_(*nii)]
    return out


def naive_field(psi0: np.ndarray, dx, t: float, lam, a=None, abar=None) -> np.ndarray:
    """The naive magnified DFT of Sec. 4.3 (eq. Psinaive), 1-D or d-D.

    One FFT, the coarse-lattice free-flight phase with the offset abar, and one
    inverse FFT read at n'' = (nbar lam) mod M.  The overall scale factor the
    paper inserts by hand is left out (taken as 1): the negative test compares
    shapes after the best complex scale fit, so it cannot matter.  The map is
    wrong once the cloud outgrows the box; it exists only as a negative test."""
    psi = np.asarray(psi0).astype(np.complex128)
    dims = psi.shape
    d = len(dims)
    dx = _as_tuple(dx, d, "dx")
    lam = tuple(int(v) for v in _as_tuple(lam, d, "lam"))
    a = _as_tuple(a, d, "a") if a is not None else tuple(default_a(dims[j], dx[j]) for j in range(d))
    if abar is None:
        abar = tuple(default_abar(dims[j], dx[j], lam[j], a[j]) for j in range(d))
    else:
        abar = _as_tuple(abar, d, "abar")
    A = np.fft.fftn(psi)
    ph = np.zeros(dims)
    for j in range(d):
        s = [1] * d
        s[j] = dims[j]
        kj = (2 * np.pi / (dims[j] * dx[j]) * symmetric_index(dims[j])).reshape(s)
        # psi-tilde carries exp(-i a k) (eq. Psiwtm); the naive inverse uses exp(+i abar k)
        ph = ph + kj * (abar[j] - a[j]) - 0.5 * t * kj * kj
    B = np.fft.ifftn(A * np.exp(1j * ph))
    nii = [np.mod(np.arange(dims[j]) * lam[j], dims[j]) for j in range(d)]
    return B[np.ix_(*nii)]


def far_field_density(psi0: np.ndarray, dx, t: float, xbar_axes) -> np.ndarray:
    """Far-field estimate rho_ff(r) = t^-d |psi~(r / t)|^2 (eq. farfieldk, hbar=m=1).

    psi~(kappa) = (2 pi)^(-d/2) sum_n dV psi_n exp(-i kappa . x_n) is the
    continuous transform (eq. FT) of the lattice field, evaluated directly at
    kappa = xbar / t on the given output axes (a list of 1-D arrays)."""
    psi = np.asarray(psi0).astype(np.complex128)
    dims = psi.shape
    d = len(dims)
    dx = _as_tuple(dx, d, "dx")
    a = [default_a(dims[j], dx[j]) for j in range(d)]
    v = psi
    for j in range(d):
        x = a[j] + np.arange(dims[j]) * dx[j]
        kappa = np.asarray(xbar_axes[j], np.float64) / t
        E = np.exp(-1j * kappa[:, None] * x[None, :]) * dx[j] / np.sqrt(2 * np.pi)
        v = _apply_along(E, v, j)
    return np.abs(v) ** 2 / t ** d
