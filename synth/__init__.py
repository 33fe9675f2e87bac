"""Seeded synthetic orbital sets shaped like the paper's workloads.

This module only draws random numbers and evaluates band-limited Gaussian
sums on a periodic grid.  It holds none of the exchange method's arithmetic
(no orthonormalisation, localisation, screening, Poisson solve or ACE step):
both the FP64 oracle and the CUDA library receive the arrays it returns and
do every step of the method themselves.

The paper's systems (amorphous silica, C3OG in water, a TiO2 cluster; Sec. 4)
are not available; these generators stand in for their shapes: orthorhombic
cells of 10-40 bohr, hundreds of occupied orbitals, 24-128 point grids, and
orbitals that are smooth (band-limited to |G|^2/2 < E_cut, the plane-wave
cutoff of Sec. 3) and localisable (built around atom-like centres, then
mixed by a random orthogonal matrix so that they start delocalised like
canonical Kohn-Sham orbitals).

Conventions: Hartree atomic units, Gamma point, real orbitals, layout
``[n_orb][n1][n2][n3]`` C-order (z fastest), float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "System",
    "fft_frequencies",
    "bandlimited_gaussian_sums",
    "config1_plain",
    "config2_water_like",
    "config3_water_like_with_extras",
    "small_localized_system",
    "random_orthogonal",
    "ServingSystem",
    "serving_systems",
    "serving_orbitals",
    "perturb_in_place",
    "batch_instances",
]


@dataclass
class System:
    """One synthetic input: a cell, a grid and raw (not orthonormal) orbitals."""

    cell: tuple[float, float, float]
    shape: tuple[int, int, int]
    ecut: float
    phi: np.ndarray  # (n_occ + n_extra, n1, n2, n3) float64, raw
    n_occ: int
    n_extra: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)


def fft_frequencies(n: int, length: float) -> np.ndarray:
    """Reciprocal-lattice components 2*pi*m/length with m in FFT order."""
    m = np.fft.fftfreq(n, d=1.0 / n)  # 0..ceil(n/2)-1, -floor(n/2)..-1
    return 2.0 * np.pi * m / length


def bandlimited_gaussian_sums(cell, shape, ecut, centers, alphas, coefs, owner, n_orb):
    """Evaluate periodic Gaussian sums truncated to |G|^2/2 < ecut on the grid.

    Term t contributes coefs[t] * exp(-alphas[t] |r - centers[t]|^2) to
    orbital owner[t].  Its Fourier coefficient is
    coefs * (pi/alpha)^{3/2} / Omega * exp(-G^2 / (4 alpha)) * exp(-i G.R);
    coefficients outside the cutoff sphere are dropped and the rest are
    transformed back to the real-space grid.  The sphere must not reach the
    Nyquist planes, so the result is exactly real up to rounding.
    """
    a, b, c = cell
    n1, n2, n3 = shape
    omega = a * b * c
    gx, gy, gz = fft_frequencies(n1, a), fft_frequencies(n2, b), fft_frequencies(n3, c)
    g2 = gx[:, None, None] ** 2 + gy[None, :, None] ** 2 + gz[None, None, :] ** 2
    mask = g2 / 2.0 < ecut
    for ax, (n, g) in enumerate(((n1, gx), (n2, gy), (n3, gz))):
        if n % 2 == 0:
            nyq = np.abs(g).max()
            if nyq * nyq / 2.0 < ecut:
                raise ValueError(f"cutoff sphere reaches the Nyquist plane on axis {ax}")
    out = np.zeros((n_orb, n1, n2, n3), dtype=np.float64)
    for o in range(n_orb):
        terms = np.nonzero(owner == o)[0]
        coef = np.zeros((n1, n2, n3), dtype=np.complex128)
        for t in terms:
            al = alphas[t]
            R = centers[t]
            amp = coefs[t] * (np.pi / al) ** 1.5 / omega
            ph = (np.exp(-1j * gx * R[0])[:, None, None]
                  * np.exp(-1j * gy * R[1])[None, :, None]
                  * np.exp(-1j * gz * R[2])[None, None, :])
            coef += amp * np.exp(-g2 / (4.0 * al)) * ph
        coef *= mask
        # f(r_m) = sum_G coef(G) e^{iG.r_m}  ==  Ng * ifftn(coef)
        out[o] = np.real(np.fft.ifftn(coef)) * (n1 * n2 * n3)
    return out


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian matrix, sign-fixed)."""
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))[None, :]


def _gaussian_terms(rng, centers_of_orbital, n_terms, jitter):
    n_orb = len(centers_of_orbital)
    owner = np.repeat(np.arange(n_orb), n_terms)
    base = np.repeat(centers_of_orbital, n_terms, axis=0)
    centers = base + (rng.normal(0.0, jitter, size=base.shape) if jitter > 0 else 0.0)
    alphas = rng.uniform(0.5, 2.0, size=len(owner))
    coefs = rng.uniform(-1.0, 1.0, size=len(owner))
    return centers, alphas, coefs, owner


def config1_plain(seed: int = 1801 + 0) -> System:
    """Plain exchange workload: cubic L=10 bohr, 24^3, 8 orbitals of 4 Gaussians.

    Each orbital is a sum of 4 s-type Gaussians (exponents U[0.5,2] bohr^-2,
    coefficients U[-1,1]) at independent uniform centres, band-limited to
    |G|^2/2 < 20 Ha.  Returned raw; orthonormalisation is the method's job.
    """
    rng = np.random.default_rng(seed)
    L, n, N, ecut = 10.0, 24, 8, 20.0
    owner = np.repeat(np.arange(N), 4)
    centers = rng.uniform(0.0, L, size=(len(owner), 3))
    alphas = rng.uniform(0.5, 2.0, size=len(owner))
    coefs = rng.uniform(-1.0, 1.0, size=len(owner))
    phi = bandlimited_gaussian_sums((L, L, L), (n, n, n), ecut, centers, alphas, coefs, owner, N)
    return System((L, L, L), (n, n, n), ecut, phi, N, 0, seed, {"name": "plain-8orb-24^3"})


def _water_like(rng, cell, shape, ecut, n_centres, n_occ, mix=True):
    centres = rng.uniform(0.0, 1.0, size=(n_centres, 3)) * np.asarray(cell)[None, :]
    owner_centre = np.arange(n_occ) % n_centres
    centers, alphas, coefs, owner = _gaussian_terms(rng, centres[owner_centre], 4, 0.5)
    phi = bandlimited_gaussian_sums(cell, shape, ecut, centers, alphas, coefs, owner, n_occ)
    if mix:
        q = random_orthogonal(n_occ, rng)
        phi = np.tensordot(q.T, phi, axes=(1, 0))
    return phi


def config2_water_like(seed: int = 1801 + 1, shape=(72, 72, 72)) -> System:
    """Localised-exchange workload shaped like a 64-molecule water box.

    Cubic L=23.5 bohr, 192 O-like centres uniform in the cell, 256 orbitals.
    Orbital o is 4 Gaussians at centre (o mod 192) displaced by N(0, 0.5^2)
    per axis, band-limited to E_cut=40 Ha, then all orbitals are mixed by one
    random orthogonal matrix (delocalised like canonical orbitals).  Raw.
    """
    rng = np.random.default_rng(seed)
    L = 23.5
    cell = (L, L, L)
    phi = _water_like(rng, cell, shape, 40.0, 192, 256)
    return System(cell, tuple(shape), 40.0, phi, 256, 0, seed, {"name": f"water-like-256orb-{shape[0]}^3"})


def config3_water_like_with_extras(seed: int = 1801 + 2, shape=(96, 96, 96)) -> System:
    """ACE workload: the water-like system with 256 occupied + 128 extra orbitals.

    The extra orbitals follow the same recipe on 128 fresh random centres and
    are returned raw; the method orthonormalises them against the occupied
    set.
    """
    rng = np.random.default_rng(seed)
    L = 23.5
    cell = (L, L, L)
    occ = _water_like(rng, cell, shape, 40.0, 192, 256)
    extra = _water_like(rng, cell, shape, 40.0, 128, 128, mix=False)
    phi = np.concatenate([occ, extra], axis=0)
    return System(cell, tuple(shape), 40.0, phi, 256, 128, seed, {"name": f"water-like-256+128orb-{shape[0]}^3"})


def small_localized_system(seed: int, cell, shape, ecut, n_centres, n_occ, n_extra=0, mix=True) -> System:
    """Scaled-down water-like system for parity tests (same recipe, any size)."""
    rng = np.random.default_rng(seed)
    occ = _water_like(rng, cell, shape, ecut, n_centres, n_occ, mix=mix)
    if n_extra:
        extra = _water_like(rng, cell, shape, ecut, max(1, n_extra), n_extra, mix=False)
        phi = np.concatenate([occ, extra], axis=0)
    else:
        phi = occ
    return System(tuple(cell), tuple(shape), ecut, phi, n_occ, n_extra, seed,
                  {"name": f"small-{n_occ}+{n_extra}orb-{shape[0]}x{shape[1]}x{shape[2]}"})


# ------------------------------------------------------------------ serving workload

def _smooth_235(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


SERVING_SIZES = tuple(n for n in range(48, 129) if _smooth_235(n))
WATER_BOHR3_PER_ORBITAL = 30.0 * 1.8897261**3 / 4.0  # 30 A^3 per molecule, 4 occupied orbitals


@dataclass
class ServingSystem:
    """One resident system of the serving stream (orbitals made on demand)."""

    index: int
    cell: tuple[float, float, float]
    shape: tuple[int, int, int]
    ecut: float
    n_occ: int
    seed: int


def serving_systems(seed: int = 1801 + 4, n_systems: int = 32) -> list[ServingSystem]:
    """Resident systems of the serving stream: N log-uniform in [32, 512],
    cubic grids drawn from the 2/3/5-smooth sizes in [48, 128], water
    density (cell volume N x 30 A^3 / 4), cutoff min(40 Ha, 0.45 (pi n / L)^2)
    so the band limit stays inside the grid's Nyquist cube."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_systems):
        n_occ = int(round(np.exp(rng.uniform(np.log(32), np.log(512)))))
        n = int(rng.choice(SERVING_SIZES))
        L = float((n_occ * WATER_BOHR3_PER_ORBITAL) ** (1.0 / 3.0))
        ecut = float(min(40.0, 0.45 * (np.pi * n / L) ** 2))
        out.append(ServingSystem(k, (L, L, L), (n, n, n), ecut, n_occ, int(rng.integers(1 << 31))))
    return out


def _periodic_gaussian_1d(n: int, L: float, ecut: float, centres: np.ndarray, alphas: np.ndarray) -> np.ndarray:
    """Rows t: sqrt(pi/alpha_t)/L * sum_{G^2/2 < ecut} exp(-G^2/(4 alpha_t)) cos(G (x - X_t)) on the n grid
    points of [0, L): the 1D factor of a Gaussian band-limited to a cube."""
    x = np.arange(n) * (L / n)
    mmax = int(np.floor(np.sqrt(2.0 * ecut) * L / (2.0 * np.pi) - 1e-12))
    if mmax >= n // 2:
        raise ValueError("band limit reaches the Nyquist plane")
    G = 2.0 * np.pi * np.arange(1, mmax + 1) / L
    d = x[None, :] - centres[:, None]                                   # (t, n)
    w = np.exp(-G[None, :] ** 2 / (4.0 * alphas[:, None]))              # (t, m)
    s = 1.0 + 2.0 * np.einsum("tm,tmn->tn", w, np.cos(G[None, :, None] * d[:, None, :]))
    return s * (np.sqrt(np.pi / alphas) / L)[:, None]


def serving_orbitals(s: ServingSystem, out: np.ndarray | None = None) -> np.ndarray:
    """Raw orbitals of a serving system, [n_occ][n][n][n] float64: orbital o is
    4 Gaussians (alpha ~ U[0.5, 2], c ~ U[-1, 1]) around centre o mod N_c
    (N_c = 3N/4 uniform centres, N(0, 0.5^2) jitter), band-limited to the
    cube |G_a|^2/2 < E_cut so that every term is a product of 1D factors.
    Not mixed: the orbitals start localised.  `out` (optional) receives them."""
    rng = np.random.default_rng(s.seed)
    n, L, N = s.shape[0], s.cell[0], s.n_occ
    n_c = max(1, (3 * N) // 4)
    centres = rng.uniform(0.0, L, size=(n_c, 3))
    owner = np.repeat(np.arange(N), 4)
    pos = centres[owner % n_c] + rng.normal(0.0, 0.5, size=(4 * N, 3))
    alphas = rng.uniform(0.5, 2.0, size=4 * N)
    coefs = rng.uniform(-1.0, 1.0, size=4 * N)
    f = [_periodic_gaussian_1d(n, L, s.ecut, pos[:, a], alphas) for a in range(3)]
    if out is None:
        out = np.empty((N, n, n, n), dtype=np.float64)
    assert out.shape == (N, n, n, n) and out.dtype == np.float64 and out.flags.c_contiguous
    fx = (f[0] * coefs[:, None]).reshape(N, 4, n)
    fy, fz = f[1].reshape(N, 4, n), f[2].reshape(N, 4, n)
    for o in range(N):
        xy = np.ascontiguousarray((fx[o][:, :, None] * fy[o][:, None, :]).reshape(4, n * n).T)  # (n^2, 4)
        np.matmul(xy, fz[o], out=out[o].reshape(n * n, n))
    return out


def perturb_in_place(phi: np.ndarray, eps: float) -> None:
    """One SCF-like step of drift: phi_o += eps * T phi_{(o+1) mod N}, T a
    shift by one grid point along x (band-limited, and out of the current
    span, so E_x moves; orthonormalisation is the method's job)."""
    first = np.roll(phi[0], 1, axis=0)
    for o in range(len(phi) - 1):
        phi[o] += eps * np.roll(phi[o + 1], 1, axis=0)
    phi[-1] += eps * first


# ------------------------------------------------------------------ batched uneven instances

BATCH_SIZES = tuple(n for n in range(32, 65) if _smooth_235(n))


def batch_instances(seed: int = 1801 + 3, n_instances: int = 48) -> list[ServingSystem]:
    """Independent cubic cells for the batched workload: L ~ U[10, 20] bohr,
    grids drawn from the 2/3/5-smooth sizes in [32, 64], N log-uniform in
    [16, 128], cutoff min(40 Ha, 0.45 (pi n / L)^2) (band limit inside the
    Nyquist cube).  Orbitals: serving_orbitals (cube band limit, localised)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        L = float(rng.uniform(10.0, 20.0))
        n = int(rng.choice(BATCH_SIZES))
        n_occ = int(round(np.exp(rng.uniform(np.log(16), np.log(128)))))
        ecut = float(min(40.0, 0.45 * (np.pi * n / L) ** 2))
        out.append(ServingSystem(k, (L, L, L), (n, n, n), ecut, n_occ, int(rng.integers(1 << 31))))
    return out
