"""Seeded synthetic initial fields for the free-flight expansion.

This module only draws and shapes initial wavefunctions psi0 and states the
lattice/flight parameters of each workload.  It holds none of the expansion's
arithmetic, so both the CUDA path's tests and the FP64 oracle's tests can take
their inputs from it without sharing any method code.

The paper's own initial states come from stochastic / Gross-Pitaevskii
simulations of the Vienna experiments (Sec. 3 eq. SGPE; Sec. 6 eqs. 3dic, GPE)
that are not available here.  Seeded fields with the same structure stand in
for them: Thomas-Fermi envelopes with dark solitons (defect-laden
quasicondensates, Sec. 3), thermal axial phase fluctuations, and a pair of
clouds with a random relative phase (the interferometer, Sec. 6).

Conventions (units hbar = m = 1):
  * realization r of a workload draws from numpy ``default_rng(seed + r)``;
  * fields are generated in float64 and rounded to complex64;
  * lattice axis j has x_n = a_j + n dx_j with a_j = -L_j/2;
  * a Gaussian of width sigma has amplitude exp(-(x - c)^2 / (2 sigma^2));
  * "TF" is sqrt(max(0, 1 - sum_j (x_j / R_j)^2)) with peak amplitude 1;
  * a dark soliton at x_k of width w multiplies by tanh((x - x_k) / w).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "axis_coords",
    "tf_soliton_1d",
    "two_cloud_3d",
    "quasicondensate_3d",
    "config_1d",
    "config_two_cloud",
    "config_quasicondensate",
    "config_mixed_batch",
    "config_large",
    "WORKLOADS",
]


@dataclass
class Workload:
    """One expansion problem: lattice, magnification, flight time, inputs."""

    name: str
    dims: tuple            # lattice points per axis (row-major, last axis contiguous)
    dx: tuple              # spacing per axis
    lam: tuple             # integer magnification per axis
    t: float               # flight time (hbar t / m)
    batch: int             # realizations
    seed: int
    make: object = field(repr=False, default=None)   # make(rng) -> complex128 array[dims]
    fringe: tuple | None = None  # interferometers: (separation axis, cloud separation D)

    def realization(self, r: int) -> np.ndarray:
        """Realization r as complex64 (drawn in float64, then rounded)."""
        rng = np.random.default_rng(self.seed + r)
        return np.asarray(self.make(rng), dtype=np.complex128).astype(np.complex64)

    def batch_array(self, count: int | None = None, start: int = 0) -> np.ndarray:
        """Realizations start..start+count-1 stacked as complex64 [count, *dims]."""
        count = self.batch if count is None else count
        out = np.empty((count,) + tuple(self.dims), np.complex64)
        for i in range(count):
            out[i] = self.realization(start + i)
        return out


def axis_coords(N: int, dx: float) -> np.ndarray:
    """Lattice coordinates x_n = -L/2 + n dx."""
    return -0.5 * N * dx + dx * np.arange(N, dtype=np.float64)


def _grids(dims, dx):
    axes = [axis_coords(n, h) for n, h in zip(dims, dx)]
    return np.meshgrid(*axes, indexing="ij")


def tf_soliton_1d(rng, N=512, dx=0.1, R=20.0, n_sol=3, span=12.0, width=0.5):
    """1-D Thomas-Fermi amplitude times n_sol dark solitons at seeded positions."""
    x = axis_coords(N, dx)
    psi = np.sqrt(np.maximum(0.0, 1.0 - (x / R) ** 2))
    for xk in rng.uniform(-span, span, size=n_sol):
        psi = psi * np.tanh((x - xk) / width)
    return psi.astype(np.complex128)


def two_cloud_3d(rng, dims=(64, 64, 64), dx=(0.25, 0.25, 0.25),
                 sigma=(2.0, 2.0, 8.0), centre=6.0):
    """Two elongated Gaussian clouds at x = -centre and x = +centre with a
    seeded relative phase phi ~ U[0, 2 pi): g(x - c) + exp(i phi) g(x + c)."""
    X, Y, Z = _grids(dims, dx)
    phi = rng.uniform(0.0, 2.0 * np.pi)
    sy = (Y / sigma[1]) ** 2 + (Z / sigma[2]) ** 2
    g1 = np.exp(-0.5 * (((X - centre) / sigma[0]) ** 2 + sy))
    g2 = np.exp(-0.5 * (((X + centre) / sigma[0]) ** 2 + sy))
    return g1 + np.exp(1j * phi) * g2


def quasicondensate_3d(rng, dims=(32, 32, 512), dx=(0.25, 0.25, 0.5),
                       radii=(3.0, 3.0, 100.0), n_modes=256, T=0.05,
                       max_solitons=4, span=60.0, width=0.5):
    """Elongated quasicondensate: TF envelope times exp(i theta(z)) times
    0..max_solitons planar dark solitons along z.

    theta(z) = sum_{n=1}^{n_modes} a_n cos(k_n z) + b_n sin(k_n z),
    k_n = 2 pi n / L_z, a_n, b_n ~ Normal(0, T / k_n^2) (thermal phase)."""
    X, Y, Z = _grids(dims, dx)
    env = np.sqrt(np.maximum(0.0, 1.0 - (X / radii[0]) ** 2 - (Y / radii[1]) ** 2
                             - (Z / radii[2]) ** 2))
    Lz = dims[2] * dx[2]
    z = axis_coords(dims[2], dx[2])
    kn = 2.0 * np.pi * np.arange(1, n_modes + 1) / Lz
    sd = np.sqrt(T) / kn
    an = rng.normal(0.0, 1.0, n_modes) * sd
    bn = rng.normal(0.0, 1.0, n_modes) * sd
    theta = np.cos(np.outer(z, kn)) @ an + np.sin(np.outer(z, kn)) @ bn
    ns = int(rng.integers(0, max_solitons + 1))
    sol = np.ones_like(z)
    for zk in rng.uniform(-span, span, size=ns):
        sol = sol * np.tanh((z - zk) / width)
    axial = np.exp(1j * theta) * sol
    return env * axial[None, None, :]


# ---------------------------------------------------------------------------
# the workloads of the benchmark and the tests
# ---------------------------------------------------------------------------

def config_1d(seed: int = 1) -> Workload:
    """1-D: N=512, dx=0.1, TF(R=20) x 3 solitons in [-12, 12], lam=20, t=40."""
    return Workload("1d_tf_solitons_N512_lam20", (512,), (0.1,), (20,), 40.0, 1, seed,
                    lambda rng: tf_soliton_1d(rng))


def config_two_cloud(seed: int = 2, batch: int = 1) -> Workload:
    """3-D interferometer: 64^3, dx=0.25, sigma=(2,2,8), centres +-6 along x,
    lam=(30,30,3), t=40."""
    return Workload("3d_two_cloud_64^3_lam30x30x3", (64, 64, 64), (0.25, 0.25, 0.25),
                    (30, 30, 3), 40.0, batch, seed, lambda rng: two_cloud_3d(rng), fringe=(0, 12.0))


def config_quasicondensate(seed: int = 3, batch: int = 256) -> Workload:
    """3-D quasicondensate ensemble: 32x32x512, dx=(0.25,0.25,0.5),
    TF(3,3,100), 256 thermal axial modes (T=0.05), 0-4 solitons;
    lam=(50,50,5), t=40, 256 realizations (mean density)."""
    return Workload("3d_quasicondensate_32x32x512_lam50x50x5", (32, 32, 512),
                    (0.25, 0.25, 0.5), (50, 50, 5), 40.0, batch, seed,
                    lambda rng: quasicondensate_3d(rng))


MIXED_SHAPES = ((48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 32, 32))


def config_mixed_batch(seed: int = 4, count: int = 1000):
    """Mixed batch: ``count`` instances, lattice drawn uniformly from
    MIXED_SHAPES, dx=0.25, two-cloud geometry scaled per axis by L_j/16
    (sigma=(L_x/8, L_y/8, L_z/2), centres +-3 L_x/8), isotropic integer
    lam ~ U{10..100}, t = 4 lam.  Returns a list of Workload (batch 1 each)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dims = MIXED_SHAPES[int(rng.integers(0, len(MIXED_SHAPES)))]
        lam = int(rng.integers(10, 101))
        L = tuple(n * 0.25 for n in dims)
        sigma = (L[0] / 8, L[1] / 8, L[2] / 2)
        centre = 3 * L[0] / 8
        out.append(Workload(f"mixed_{i}", dims, (0.25,) * 3, (lam,) * 3, 4.0 * lam, 1,
                            seed * 100003 + i,
                            (lambda d, s, c: (lambda r: two_cloud_3d(r, d, (0.25,) * 3, s, c)))(
                                dims, sigma, centre)))
    return out


def config_large(which: str = "two_cloud", seed: int = 5) -> Workload:
    """Large 3-D cases with lam=100 on every axis and t=400:
    ``two_cloud``: 256^3, dx=0.25 (L=64), sigma=(2,2,8), centres +-6;
    ``quasicondensate``: 128x128x1024, dx=(0.25,0.25,0.5), TF(3,3,100),
    256 axial modes with k_n = 2 pi n / 512."""
    if which == "two_cloud":
        return Workload("3d_two_cloud_256^3_lam100", (256, 256, 256), (0.25,) * 3,
                        (100, 100, 100), 400.0, 1, seed,
                        lambda rng: two_cloud_3d(rng, (256, 256, 256)), fringe=(0, 12.0))
    if which == "quasicondensate":
        return Workload("3d_quasicondensate_128x128x1024_lam100", (128, 128, 1024),
                        (0.25, 0.25, 0.5), (100, 100, 100), 400.0, 1, seed,
                        lambda rng: quasicondensate_3d(rng, (128, 128, 1024)))
    raise ValueError(which)


WORKLOADS = {
    "1d": config_1d,
    "two_cloud": config_two_cloud,
    "quasicondensate": config_quasicondensate,
    "large_two_cloud": lambda: config_large("two_cloud"),
    "large_quasicondensate": lambda: config_large("quasicondensate"),
}
