"""Plain FP64 CPU oracle of the L-ACE exchange hot path (arXiv:1801.09263).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module.  The CUDA library
never calls it and shares no code with it.

Every function states the passage of the paper it follows.  Conventions
(where the paper is silent, the reading taken):

* Hartree atomic units with e^2 = 1; Gamma point; real orbitals.
* The paper's V_X carries a minus sign to be positive definite (Sec. 2,
  after Eq. 1).  Here K = -V_X is the physical exchange operator, negative
  semidefinite, so M = Psi^T K Psi = -L L^T and K psi ~= -xi (xi^T psi).
* Grid of n1 x n2 x n3 points in an orthorhombic cell a x b x c,
  Omega = abc, Ng = n1 n2 n3, dV = Omega / Ng.  Orbitals are normalised so
  that dV * sum_r phi(r)^2 = 1.  Inner products carry dV.
* Coulomb kernel K(G) = 4 pi / |G|^2 on every G of the grid (no cutoff
  sphere), with K(0) = 0 (the G = 0 term is dropped; nothing else).  The
  erfc-screened kernel of range-separated hybrids (Grid.kernel = "erfc") is
  finite at G = 0; either kernel is scaled by the exchange fraction alpha.
* Forward FFT unscaled, inverse FFT scaled by 1/Ng (numpy convention).

The FFT (scipy.fft), symmetric eigensolver, Cholesky factorisation and
triangular solve are library primitives used as single steps.  Parity:
every function here is pinned by the not-gpu tests (brute-force sums,
closed forms, invariants, library cross-checks) except the screened L-ACE
values, which have no closed form: screened results are "parity unpinned"
beyond the self-consistency checks (L-ACE(0) == ACE, monotone kept counts).
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import scipy.fft
import scipy.linalg

__all__ = [
    "Grid",
    "coulomb_kernel",
    "screened_kernel",
    "interaction_kernel",
    "pair_potential",
    "lowdin",
    "orthonormalize_extras",
    "qrcp_pivots",
    "subsample_indices",
    "qrcp_pivot_ratios",
    "scdm",
    "overlap_moduli",
    "align_orbitals",
    "pw_basis",
    "pw_to_grid",
    "grid_to_pw",
    "kept_pairs",
    "apply_exchange",
    "apply_exchange_columns",
    "exchange_energy_gspace",
    "symmetrize",
    "ace_build",
    "ace_apply",
]

_WORKERS = max(1, len(os.sched_getaffinity(0)))


@dataclass(frozen=True)
class Grid:
    """Orthorhombic periodic cell and its real-space grid, and the interaction
    kernel of the exchange operator: "coulomb" (Eq. 2) or "erfc" (the
    short-range screened kernel of range-separated hybrids such as HSE,
    Sec. 4, with range-separation parameter `screening` (omega of HSE, in
    bohr^-1; not the cell volume omega below), scaled by the exact-exchange
    fraction alpha."""

    cell: tuple  # (a, b, c) in bohr
    shape: tuple  # (n1, n2, n3)
    kernel: str = "coulomb"
    screening: float = 0.0
    alpha: float = 1.0

    @property
    def omega(self) -> float:
        a, b, c = self.cell
        return float(a) * float(b) * float(c)

    @property
    def ng(self) -> int:
        n1, n2, n3 = self.shape
        return int(n1) * int(n2) * int(n3)

    @property
    def dv(self) -> float:
        return self.omega / self.ng


def _freq(n: int, length: float) -> np.ndarray:
    # G = 2 pi m / length with m in FFT order 0..ceil(n/2)-1, -floor(n/2)..-1
    m = np.concatenate([np.arange(0, (n + 1) // 2), np.arange(-(n // 2), 0)])
    return 2.0 * np.pi * m / length


def g_squared(grid: Grid) -> np.ndarray:
    """|G|^2 on the full FFT grid, axis order (n1, n2, n3)."""
    (a, b, c), (n1, n2, n3) = grid.cell, grid.shape
    gx, gy, gz = _freq(n1, a), _freq(n2, b), _freq(n3, c)
    return gx[:, None, None] ** 2 + gy[None, :, None] ** 2 + gz[None, None, :] ** 2


def coulomb_kernel(grid: Grid) -> np.ndarray:
    """K(G) = 4 pi e^2 / |G|^2 with K(0) = 0 (Eq. 2 in reciprocal space, Sec. 2).

    The paper solves the integrals of Eq. 2 with FFTs on the exchange grid;
    it does not treat the G = 0 divergence specially, so the term is dropped.
    """
    g2 = g_squared(grid)
    k = np.zeros_like(g2)
    nz = g2 > 0
    k[nz] = 4.0 * np.pi / g2[nz]
    return k


def screened_kernel(grid: Grid, omega: float) -> np.ndarray:
    """K(G) = 4 pi / |G|^2 (1 - exp(-|G|^2 / (4 omega^2))), K(0) = pi / omega^2.

    The Fourier transform of erfc(omega r) / r, the short-range part of the
    Coulomb interaction that range-separated hybrids such as HSE keep in the
    exact exchange (the paper applies L-ACE to HSE in Sec. 4 without giving
    the kernel; this is the standard one).  Finite at G = 0: the limit of
    4 pi (1 - exp(-x)) / |G|^2 with x = |G|^2 / (4 omega^2) is pi / omega^2.
    """
    g2 = g_squared(grid)
    k = np.empty_like(g2)
    nz = g2 > 0
    k[nz] = 4.0 * np.pi / g2[nz] * -np.expm1(-g2[nz] / (4.0 * omega * omega))
    k[~nz] = np.pi / (omega * omega)
    return k


def interaction_kernel(grid: Grid) -> np.ndarray:
    """The grid's kernel: coulomb_kernel or screened_kernel, times alpha."""
    if grid.kernel == "coulomb":
        k = coulomb_kernel(grid)
    elif grid.kernel == "erfc":
        k = screened_kernel(grid, grid.screening)
    else:
        raise ValueError(f"unknown kernel {grid.kernel!r}")
    return k * grid.alpha if grid.alpha != 1.0 else k


def pair_potential(grid: Grid, rho: np.ndarray) -> np.ndarray:
    """Potential of a (batch of) real pair densities: v = IFFT(K * FFT(rho)).

    This is the inner integral of Eq. 2, int dr' rho(r') / |r - r'|, evaluated
    with FFTs as the paper describes for plane waves (Sec. 2).  rho has shape
    (..., n1, n2, n3).
    """
    k = interaction_kernel(grid)
    n1, n2, n3 = grid.shape
    kh = k[:, :, : n3 // 2 + 1]  # real-to-complex half spectrum
    axes = (-3, -2, -1)
    rg = scipy.fft.rfftn(rho, axes=axes, workers=_WORKERS)
    return scipy.fft.irfftn(rg * kh, s=(n1, n2, n3), axes=axes, workers=_WORKERS)


def lowdin(grid: Grid, phi: np.ndarray) -> np.ndarray:
    """Symmetric (Loewdin) orthonormalisation: phi <- phi S^{-1/2}, S = dV phi^T phi.

    The paper works with orthonormal Kohn-Sham orbitals (Sec. 2); the
    inputs here are raw Gaussian sums, so they are orthonormalised first.
    S^{-1/2} comes from the symmetric eigendecomposition of S.
    """
    n = phi.shape[0]
    a = phi.reshape(n, -1)
    s = grid.dv * (a @ a.T)
    lam, vec = np.linalg.eigh(s)
    if lam.min() <= 1e-12 * lam.max():
        raise np.linalg.LinAlgError("overlap matrix is singular or ill-conditioned")
    x = (vec * (1.0 / np.sqrt(lam))[None, :]) @ vec.T
    return (x.T @ a).reshape(phi.shape)  # new_k = sum_j phi_j X_jk


def orthonormalize_extras(grid: Grid, occ: np.ndarray, extra: np.ndarray) -> np.ndarray:
    """Extra (virtual-like) orbitals made orthonormal to the occupied set.

    Sec. 4.1 adds virtual orbitals to the projection set N_P; they must be
    orthogonal to the occupied manifold.  Project out the (orthonormal)
    occupied orbitals once, then Loewdin-orthonormalise what is left.
    """
    no, ne = occ.shape[0], extra.shape[0]
    o = occ.reshape(no, -1)
    e = extra.reshape(ne, -1)
    c = grid.dv * (o @ e.T)  # (no, ne) overlaps
    e = e - c.T @ o
    return lowdin(grid, e.reshape(extra.shape))


def subsample_indices(shape, stride: int = 2) -> np.ndarray:
    """Linear full-grid indices of the points whose three indices are multiples of stride."""
    n1, n2, n3 = shape
    i = np.arange(0, n1, stride)
    j = np.arange(0, n2, stride)
    k = np.arange(0, n3, stride)
    return ((i[:, None, None] * n2 + j[None, :, None]) * n3 + k[None, None, :]).ravel()


def qrcp_pivots(a: np.ndarray, n_piv: int | None = None) -> np.ndarray:
    """Column pivots of a QR factorisation with column pivoting (Businger-Golub).

    SCDM (Sec. 2, ref. Damle et al.) selects the columns of the density
    matrix by a pivoted QR of the orbital matrix.  Step by step: take the
    remaining column with the largest residual 2-norm (ties: lowest column
    index), normalise it, and remove its direction from every column
    (modified Gram-Schmidt).  Norms are recomputed exactly at every step.
    a is (rows, columns); returns n_piv column indices in selection order.
    """
    r = np.array(a, dtype=np.float64, copy=True)
    nrow, ncol = r.shape
    n_piv = min(nrow, ncol) if n_piv is None else n_piv
    chosen = np.zeros(ncol, dtype=bool)
    piv = np.empty(n_piv, dtype=np.int64)
    for step in range(n_piv):
        norms = np.einsum("ij,ij->j", r, r)
        norms[chosen] = -1.0
        p = int(np.argmax(norms))  # first maximum = lowest index on ties
        piv[step] = p
        chosen[p] = True
        q = r[:, p] / np.sqrt(norms[p])
        r -= np.outer(q, q @ r)
    return piv


def qrcp_pivot_ratios(a: np.ndarray, pivots) -> np.ndarray:
    """Replay the pivoted QR of qrcp_pivots with a given pivot order.

    For every step k returns ||r_{p_k}||^2 / max_c ||r_c||^2 over the columns
    not yet chosen, with the residuals of the same exact Gram-Schmidt steps.
    A valid Businger-Golub pivot order has every ratio equal to 1; a ratio
    slightly below 1 marks a choice between near-tied columns.
    """
    r = np.array(a, dtype=np.float64, copy=True)
    chosen = np.zeros(r.shape[1], dtype=bool)
    out = np.empty(len(pivots))
    for step, p in enumerate(pivots):
        norms = np.einsum("ij,ij->j", r, r)
        norms[chosen] = -1.0
        out[step] = norms[p] / norms.max()
        chosen[p] = True
        q = r[:, p] / np.sqrt(norms[p])
        r -= np.outer(q, q @ r)
    return out


def scdm(grid: Grid, phi: np.ndarray, stride: int = 2, pivots=None):
    """SCDM localisation of an orthonormal occupied set (Sec. 2).

    1. Subsample the grid (every stride-th point along each axis).
    2. Pivoted QR of phi restricted to the subsample (orbitals x points)
       selects N points C.
    3. phi_C = phi at the selected points (N points x N orbitals, full grid
       values); U = phi_C^T (phi_C phi_C^T)^{-1/2}, an orthogonal matrix.
    4. Localised orbitals w = phi U.
    The paper's "modified" SCDM is not described; this is the standard one.
    If pivots is given (full-grid linear indices) the QR step is skipped.
    Returns (pivots as full-grid linear indices, U, w).
    """
    n = phi.shape[0]
    a = phi.reshape(n, -1)
    if pivots is None:
        sub = subsample_indices(grid.shape, stride)
        piv_sub = qrcp_pivots(a[:, sub], n)
        pivots = sub[piv_sub]
    pivots = np.asarray(pivots, dtype=np.int64)
    phic = a[:, pivots].T  # (points, orbitals)
    b = phic @ phic.T
    lam, vec = np.linalg.eigh(b)
    if lam.min() <= 1e-12 * lam.max():
        raise np.linalg.LinAlgError("selected columns are rank deficient")
    b_mhalf = (vec * (1.0 / np.sqrt(lam))[None, :]) @ vec.T
    u = phic.T @ b_mhalf  # (orbitals, orbitals), orthogonal
    w = (u.T @ a).reshape(phi.shape)  # w_m = sum_k phi_k U_km
    return pivots, u, w


def align_orbitals(grid: Grid, w: np.ndarray, w_prev: np.ndarray) -> tuple:
    """Rotate w within its span to the orthonormal set closest to w_prev.

    The paper improves tight SCF convergence by aligning the orbitals of an
    iteration to those of the previous one (end of Sec. 2).  Reading: the
    orthogonal Q maximising sum_j <(w Q)_j, prev_j> (orthogonal Procrustes),
    i.e. the polar factor of O = dV w prev^T, Q = U V^T from O = U S V^T
    (library SVD).  Returns (Q, aligned orbitals sum_i w_i Q_ij).
    """
    n = w.shape[0]
    a = w.reshape(n, -1)
    o = grid.dv * (a @ w_prev.reshape(n, -1).T)
    u, _, vt = np.linalg.svd(o)
    q = u @ vt
    return q, (q.T @ a).reshape(w.shape)


def pw_basis(cell, ecut: float) -> np.ndarray:
    """Plane-wave basis of real (Gamma-point) orbitals: the half sphere of
    G = 2 pi (m1/a, m2/b, m3/c) with |G|^2/2 < ecut (the orbital cutoff of
    Sec. 3), half-space m3 > 0, or m3 = 0 and m2 > 0, or m3 = m2 = 0 and
    m1 >= 0; ordered by |G|^2, ties by (m1, m2, m3).  Returns int (n_pw, 3).

    An orbital is phi(r) = c(0) + 2 Re sum_{G != 0} c(G) exp(i G.r), the
    real-orbital form of the plane-wave expansion the paper's V_X matrix is
    written in (Sec. 2)."""
    a, b, c = cell
    mm = [int(np.floor(np.sqrt(2.0 * ecut) * L / (2.0 * np.pi))) for L in (a, b, c)]
    out = []
    for m1 in range(-mm[0], mm[0] + 1):
        for m2 in range(-mm[1], mm[1] + 1):
            for m3 in range(-mm[2], mm[2] + 1):
                if not (m3 > 0 or (m3 == 0 and m2 > 0) or (m3 == 0 and m2 == 0 and m1 >= 0)):
                    continue
                g2 = (2 * np.pi * m1 / a) ** 2 + (2 * np.pi * m2 / b) ** 2 + (2 * np.pi * m3 / c) ** 2
                if g2 / 2.0 < ecut:
                    out.append((g2, m1, m2, m3))
    out.sort()
    return np.array([o[1:] for o in out], dtype=np.int64).reshape(-1, 3)


def pw_to_grid(grid: Grid, mvec: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """phi(r_j) = c(0) + 2 Re sum_{G != 0} c(G) exp(i G.r_j) on the grid:
    the full spectrum (c at G, conj(c) at -G) through the library inverse FFT.
    coef: complex (n_orb, n_pw) in pw_basis order."""
    n1, n2, n3 = grid.shape
    spec = np.zeros((coef.shape[0], n1, n2, n3), dtype=np.complex128)
    i1, i2, i3 = mvec[:, 0] % n1, mvec[:, 1] % n2, mvec[:, 2] % n3
    j1, j2, j3 = -mvec[:, 0] % n1, -mvec[:, 1] % n2, -mvec[:, 2] % n3
    zero = np.all(mvec == 0, axis=1)
    c = coef.copy()
    c[:, zero] = c[:, zero].real
    spec[:, j1, j2, j3] = np.conj(c)
    spec[:, i1, i2, i3] = c
    return np.real(np.fft.ifftn(spec, axes=(1, 2, 3))) * grid.ng


def grid_to_pw(grid: Grid, mvec: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """c(G) = (1/Ng) sum_j phi(r_j) exp(-i G.r_j) at the basis vectors."""
    n1, n2, n3 = grid.shape
    spec = np.fft.fftn(phi, axes=(1, 2, 3)) / grid.ng
    return spec[:, mvec[:, 0] % n1, mvec[:, 1] % n2, mvec[:, 2] % n3]


def overlap_moduli(grid: Grid, w: np.ndarray) -> np.ndarray:
    """S_ik = int dr |w_i(r)| |w_k(r)| on the full grid (Eq. 4)."""
    n = w.shape[0]
    aw = np.abs(w.reshape(n, -1))
    return grid.dv * (aw @ aw.T)


def kept_pairs(s: np.ndarray, s_thr: float, n_occ: int, n_extra: int) -> np.ndarray:
    """Boolean (n_occ, n_occ + n_extra) mask of the exchange integrals kept.

    Occupied-occupied pair (i, k) is dropped when S_ik < S_thr (Eq. 4 and the
    truncated potential of Eq. 5); a dropped pair removes both u^(ik) and
    u^(ki), so the mask is symmetric.  Every pair with an extra (virtual)
    orbital is kept: virtuals are not localised (Sec. 4.1).
    """
    keep = np.ones((n_occ, n_occ + n_extra), dtype=bool)
    keep[:, :n_occ] = s[:n_occ, :n_occ] >= s_thr
    return keep


def apply_exchange_columns(grid: Grid, w_occ: np.ndarray, psi: np.ndarray, keep_cols: np.ndarray):
    """K psi for a set of targets psi (Eq. 2 with the truncation of Eq. 5).

    (K psi_j)(r) = - sum_{i kept with j} w_i(r) v_ij(r),  v_ij = potential of
    the pair density w_i psi_j.  keep_cols is (n_occ, n_targets) boolean.
    Also returns the pair integrals e_ij = dV sum_r w_i psi_j v_ij (the
    exchange integrals (ij|ji) of the paper's footnote notation).
    """
    nt = psi.shape[0]
    out = np.zeros_like(psi)
    e = np.zeros((w_occ.shape[0], nt))
    chunk = 32
    for j in range(nt):
        idx = np.nonzero(keep_cols[:, j])[0]
        for s0 in range(0, len(idx), chunk):
            ii = idx[s0:s0 + chunk]
            rho = w_occ[ii] * psi[j][None]
            v = pair_potential(grid, rho)
            out[j] -= np.sum(w_occ[ii] * v, axis=0)
            e[ii, j] = grid.dv * np.sum((rho * v).reshape(len(ii), -1), axis=1)
    return out, e


def apply_exchange(grid: Grid, w_occ: np.ndarray, extras: np.ndarray | None, keep: np.ndarray,
                   f_spin: float = 1.0):
    """Exchange applied to the projection set Psi = [w_occ, extras].

    Returns (W = K Psi, E_x, pair integrals e).  E_x = 1/2 f_spin dV
    sum_{i occ} <w_i, (K w_i)> = -1/2 f_spin sum_{i,k occ, kept} e_ik (the
    exchange energy implied by Eq. 2 for unit occupations; f_spin = 2 for a
    closed shell).
    """
    psi = w_occ if extras is None or len(extras) == 0 else np.concatenate([w_occ, extras], axis=0)
    W, e = apply_exchange_columns(grid, w_occ, psi, keep)
    n_occ = w_occ.shape[0]
    ex = 0.5 * f_spin * grid.dv * float(np.sum(w_occ.reshape(n_occ, -1) * W[:n_occ].reshape(n_occ, -1)))
    return W, ex, e


def exchange_energy_gspace(grid: Grid, w_occ: np.ndarray, keep_occ: np.ndarray, f_spin: float = 1.0) -> float:
    """E_x from reciprocal space: -1/2 f sum_{kept i,k} (Omega/Ng^2) sum_G K |FFT(w_i w_k)|^2.

    Parseval form of the same energy; an independent route used by tests.
    """
    k = interaction_kernel(grid)
    n = w_occ.shape[0]
    tot = 0.0
    for i in range(n):
        for kk in range(n):
            if keep_occ[i, kk]:
                rg = np.fft.fftn(w_occ[i] * w_occ[kk])
                tot += float(np.sum(k * np.abs(rg) ** 2))
    return -0.5 * f_spin * grid.omega / grid.ng ** 2 * tot


def symmetrize(m: np.ndarray, mode: str = "avg") -> np.ndarray:
    """Symmetrisation of the truncated exchange matrix M' (Sec. 2, after Eq. 7).

    avg: (M' + M'^T)/2; upper: upper triangle copied into the lower one;
    lower: lower triangle copied into the upper one.
    """
    if mode == "avg":
        return 0.5 * (m + m.T)
    if mode == "upper":
        return np.triu(m) + np.triu(m, 1).T
    if mode == "lower":
        return np.tril(m) + np.tril(m, -1).T
    raise ValueError(mode)


def ace_build(grid: Grid, psi: np.ndarray, W: np.ndarray, sym: str = "avg"):
    """ACE projector from W = K Psi (Eq. 3 and its Cholesky form, Sec. 2).

    M = dV Psi^T W (the exchange matrix), symmetrised; -M = L L^T (Cholesky;
    M is negative definite under K = -V_X); xi = W L^{-T}.  Returns (xi, L, M).
    """
    n = psi.shape[0]
    p = psi.reshape(n, -1)
    w = W.reshape(n, -1)
    m = symmetrize(grid.dv * (p @ w.T), sym)  # M_jk = dV <psi_j, W_k>
    l = np.linalg.cholesky(-m)
    # xi_k = sum_j W_j (L^{-T})_jk  <=>  xi^T = L^{-1} W^T
    xi_t = scipy.linalg.solve_triangular(l, w, lower=True)
    return xi_t.reshape(W.shape), l, m


def ace_apply(grid: Grid, xi: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """K_ACE phi = -xi (dV xi^T phi): N_P scalar products per function (Sec. 2)."""
    n = xi.shape[0]
    x = xi.reshape(n, -1)
    f = phi.reshape(phi.shape[0], -1)
    c = grid.dv * (x @ f.T)  # (N_P, n_phi)
    return (-(c.T @ x)).reshape(phi.shape)
