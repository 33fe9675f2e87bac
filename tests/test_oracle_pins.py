"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against brute force, a closed form, an invariant
of the mathematics, or an independent library route, chosen so that a
plausible slip (dropped term, wrong sign or index, transposed operand, wrong
FFT normalisation) fails at least one of them.  No GPU is needed.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(seed=7, shape=(12, 12, 12), n_occ=6, n_extra=0, cell=(9.0, 9.0, 9.0), ecut=6.0, n_centres=4):
    sysm = synth.small_localized_system(seed, cell, shape, ecut, n_centres, n_occ, n_extra)
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi[:n_occ])
    extra = O.orthonormalize_extras(g, occ, sysm.phi[n_occ:]) if n_extra else None
    return g, occ, extra


# ---------------------------------------------------------------- Poisson / FFT


def _green_bruteforce(cell, shape, screening=None):
    """g(d) = (1/Ng) sum_G K(G) cos(G.d), by explicit sums (no FFT).

    Coulomb: K = 4 pi/|G|^2 without G = 0.  screening = w: the erfc kernel,
    K = 4 pi/|G|^2 (1 - exp(-|G|^2/(4 w^2))) written out term by term, with
    the G = 0 term pi/w^2."""
    (a, b, c), (n1, n2, n3) = cell, shape
    ng = n1 * n2 * n3
    # enumerate frequencies symmetrically; for even n take -n/2 (cos is even)
    ms = [np.arange(-(n // 2), n - n // 2) for n in shape]
    gvec = []
    for m1 in ms[0]:
        for m2 in ms[1]:
            for m3 in ms[2]:
                if m1 == 0 and m2 == 0 and m3 == 0:
                    continue
                gvec.append((2 * np.pi * m1 / a, 2 * np.pi * m2 / b, 2 * np.pi * m3 / c))
    gvec = np.array(gvec)
    g2 = np.sum(gvec ** 2, axis=1)
    kern = 4 * np.pi / g2
    if screening is not None:
        kern = kern * (1.0 - np.exp(-g2 / (4 * screening ** 2)))
        gvec = np.vstack([gvec, np.zeros(3)])
        kern = np.append(kern, np.pi / screening ** 2)
    d = np.array([(i * a / n1, j * b / n2, k * c / n3)
                  for i in range(n1) for j in range(n2) for k in range(n3)])
    return (np.cos(d @ gvec.T) @ kern / ng).reshape(shape)


def test_pair_potential_equals_bruteforce_real_space_sum():
    cell, shape = (5.0, 6.5, 7.3), (6, 8, 5)
    g = O.Grid(cell, shape)
    rng = np.random.default_rng(3)
    rho = rng.standard_normal(shape)
    green = _green_bruteforce(cell, shape)
    n1, n2, n3 = shape
    v_bf = np.zeros(shape)
    for i in range(n1):
        for j in range(n2):
            for k in range(n3):
                # v(r) = sum_r' g(r - r') rho(r'), periodic differences
                gi = green[(i - np.arange(n1)) % n1][:, (j - np.arange(n2)) % n2][:, :, (k - np.arange(n3)) % n3]
                v_bf[i, j, k] = np.sum(gi * rho)
    v = O.pair_potential(g, rho)
    assert np.max(np.abs(v - v_bf)) <= 1e-12 * np.max(np.abs(v_bf))


def test_screened_pair_potential_equals_bruteforce_sum():
    cell, shape, w = (5.0, 6.5, 7.3), (6, 8, 5), 0.7
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(shape)
    green = _green_bruteforce(cell, shape, screening=w)
    n1, n2, n3 = shape
    for alpha in (1.0, 0.25):
        g = O.Grid(cell, shape, kernel="erfc", screening=w, alpha=alpha)
        v = O.pair_potential(g, rho)
        for (i, j, k) in ((0, 0, 0), (3, 5, 2), (5, 7, 4)):
            gi = green[(i - np.arange(n1)) % n1][:, (j - np.arange(n2)) % n2][:, :, (k - np.arange(n3)) % n3]
            assert abs(v[i, j, k] - alpha * np.sum(gi * rho)) <= 1e-12 * np.max(np.abs(v))


def _erfc_self_energy(a, w):
    """(ii|ii) for phi = (a/pi)^{3/4} exp(-a r^2/2) with erfc(w r)/r, isolated:
    the separation of two points of rho = phi^2 is Gaussian with exponent
    b = a/2, <1/s> = 2 sqrt(b/pi), <erf(w s)/s> = 2 sqrt(mu/pi) with
    mu = b w^2/(b + w^2), so <erfc(w s)/s> = 2 (sqrt(b) - sqrt(mu)) / sqrt(pi)."""
    b = a / 2.0
    mu = b * w * w / (b + w * w)
    return 2.0 * (np.sqrt(b) - np.sqrt(mu)) / np.sqrt(np.pi)


@pytest.mark.parametrize("w", [0.3, 1.0])
def test_screened_gaussian_self_energy_closed_form(w):
    # short-range kernel: periodic images contribute erfc(w L)/L (< 1e-16 here),
    # and the sampled Gaussian is band-limited to exp(-25) on the 64^3 grid
    a, L, n = 1.0, 20.0, 64
    phi = _periodic_gaussian_orbital(a, L, n, centre=(0.37 * L, 0.61 * L, 0.18 * L))[None]
    keep = np.ones((1, 1), dtype=bool)
    closed = _erfc_self_energy(a, w)
    for alpha in (1.0, 0.25):
        g = O.Grid((L, L, L), (n, n, n), kernel="erfc", screening=w, alpha=alpha)
        _, ex, e = O.apply_exchange(g, phi, None, keep)
        assert abs(e[0, 0] - alpha * closed) < 1e-10
        assert abs(ex + 0.5 * alpha * closed) < 1e-10
        assert abs(O.exchange_energy_gspace(g, phi, keep) + 0.5 * alpha * closed) < 1e-10
    # w -> 0 approaches the bare Coulomb self-energy sqrt(2a/pi); the screened value is below it
    assert 0 < closed < np.sqrt(2 * a / np.pi)


def test_planted_screening_mistake_is_caught(monkeypatch):
    """exp(-|G|^2/(2 w^2)) instead of exp(-|G|^2/(4 w^2)) must fail the closed form."""
    def wrong(grid, omega):
        g2 = O.lace_oracle.g_squared(grid)
        k = np.empty_like(g2)
        nz = g2 > 0
        k[nz] = 4.0 * np.pi / g2[nz] * -np.expm1(-g2[nz] / (2.0 * omega * omega))
        k[~nz] = 2.0 * np.pi / (omega * omega)
        return k
    monkeypatch.setattr(O.lace_oracle, "screened_kernel", wrong)
    a, L, n, w = 1.0, 20.0, 48, 0.5
    phi = _periodic_gaussian_orbital(a, L, n, centre=(10.0, 10.0, 10.0))[None]
    g = O.Grid((L, L, L), (n, n, n), kernel="erfc", screening=w)
    _, _, e = O.apply_exchange(g, phi, None, np.ones((1, 1), dtype=bool))
    assert abs(e[0, 0] - _erfc_self_energy(a, w)) > 1e-3


def test_pair_potential_batch_and_odd_sizes():
    cell, shape = (4.0, 5.0, 6.0), (5, 9, 7)
    g = O.Grid(cell, shape)
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((3,) + shape)
    v = O.pair_potential(g, rho)
    green = _green_bruteforce(cell, shape)
    # one point, brute force
    i, j, k = 2, 7, 3
    n1, n2, n3 = shape
    gi = green[(i - np.arange(n1)) % n1][:, (j - np.arange(n2)) % n2][:, :, (k - np.arange(n3)) % n3]
    for b in range(3):
        assert abs(v[b, i, j, k] - np.sum(gi * rho[b])) <= 1e-12 * np.max(np.abs(v[b]))


def _periodic_gaussian_orbital(a, L, n, centre):
    """phi = (a/pi)^{3/4} exp(-a r^2 / 2), periodised, sampled on an n^3 grid."""
    x = np.arange(n) * L / n
    phi = np.zeros((n, n, n))
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                dx = (x - centre[0] + sx * L)[:, None, None]
                dy = (x - centre[1] + sy * L)[None, :, None]
                dz = (x - centre[2] + sz * L)[None, None, :]
                phi += np.exp(-a * (dx * dx + dy * dy + dz * dz) / 2)
    return (a / np.pi) ** 0.75 * phi


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "gaussian_hartree.json")))["cases"])
def test_single_gaussian_exchange_energy_closed_form(case):
    gold = json.load(open(os.path.join(GOLDEN, "gaussian_hartree.json")))
    a, L = case["a"], case["L"]
    n = 48
    phi = _periodic_gaussian_orbital(a, L, n, centre=(0.37 * L, 0.61 * L, 0.18 * L))[None]
    g = O.Grid((L, L, L), (n, n, n))
    # image overlap of the periodised orbital is exp(-a L^2/4) ~ 1e-11 at a=1, L=10
    assert abs(g.dv * np.sum(phi ** 2) - 1.0) < 1e-9
    closed = np.sqrt(2 * a / np.pi) - gold["xi_sc"] / L + 2 * np.pi / (a * L ** 3)
    keep = np.ones((1, 1), dtype=bool)
    W, ex, e = O.apply_exchange(g, phi, None, keep)
    assert abs(ex - (-0.5 * closed)) < 5e-10
    assert abs(e[0, 0] - closed) < 1e-9
    assert abs(O.exchange_energy_gspace(g, phi, keep) - (-0.5 * closed)) < 5e-10


# ---------------------------------------------------------------- orbital sets


def test_lowdin_equals_svd_polar_factor():
    sysm = synth.small_localized_system(11, (8.0, 8.0, 8.0), (10, 10, 10), 5.0, 3, 5)
    g = O.Grid(sysm.cell, sysm.shape)
    out = O.lowdin(g, sysm.phi)
    a = np.sqrt(g.dv) * sysm.phi.reshape(5, -1).T  # (points, orbitals)
    uu, _, vt = np.linalg.svd(a, full_matrices=False)
    polar = (uu @ vt).T / np.sqrt(g.dv)
    assert np.allclose(out.reshape(5, -1), polar, atol=1e-12 * np.abs(polar).max())
    s = g.dv * out.reshape(5, -1) @ out.reshape(5, -1).T
    assert np.allclose(s, np.eye(5), atol=1e-12)


def test_extras_orthogonal_to_occupied_and_span_kept():
    g, occ, extra = _small(seed=5, n_occ=5, n_extra=3)
    allp = np.concatenate([occ, extra]).reshape(8, -1)
    s = g.dv * allp @ allp.T
    assert np.allclose(s, np.eye(8), atol=1e-12)


def test_rotation_invariance_of_unscreened_exchange():
    g, occ, _ = _small(seed=21, n_occ=5)
    q = synth.random_orthogonal(5, np.random.default_rng(9))
    rot = np.tensordot(q.T, occ, axes=(1, 0))  # rot_k = sum_j occ_j Q_jk
    keep = np.ones((5, 5), dtype=bool)
    W1, ex1, _ = O.apply_exchange(g, occ, None, keep)
    W2, ex2, _ = O.apply_exchange(g, rot, None, keep)
    assert abs(ex1 - ex2) <= 1e-12 * abs(ex1)
    W1r = np.tensordot(q.T, W1, axes=(1, 0))
    assert np.max(np.abs(W1r - W2)) <= 1e-11 * np.max(np.abs(W2))


def test_exchange_operator_symmetric_and_negative_semidefinite():
    g, occ, _ = _small(seed=22, n_occ=4)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((5,) + g.shape)
    keep = np.ones((4, 5), dtype=bool)
    Kpsi, _ = O.apply_exchange_columns(g, occ, psi, keep)
    m = g.dv * psi.reshape(5, -1) @ Kpsi.reshape(5, -1).T
    assert np.max(np.abs(m - m.T)) <= 1e-12 * np.max(np.abs(m))
    lam = np.linalg.eigvalsh(0.5 * (m + m.T))
    assert lam.max() <= 1e-12 * np.abs(lam).max()
    assert lam.min() < 0


def test_energy_identity_real_space_vs_reciprocal_space_screened():
    g, occ, _ = _small(seed=23, n_occ=6)
    s = O.overlap_moduli(g, occ)
    thr = np.sort(s[np.triu_indices(6, 1)])[7]  # drop a few pairs
    keep = O.kept_pairs(s, thr, 6, 0)
    assert not keep.all() and (keep == keep.T).all()
    _, ex, e = O.apply_exchange(g, occ, None, keep)
    ex_g = O.exchange_energy_gspace(g, occ, keep)
    assert abs(ex - ex_g) <= 1e-12 * abs(ex)
    assert abs(ex - (-0.5 * np.sum(e[keep[:, :6]]))) <= 1e-12 * abs(ex)


def test_exchange_integrals_symmetric_in_pair():
    g, occ, _ = _small(seed=24, n_occ=4)
    keep = np.ones((4, 4), dtype=bool)
    _, _, e = O.apply_exchange(g, occ, None, keep)
    assert np.max(np.abs(e - e.T)) <= 1e-12 * np.max(np.abs(e))
    assert (np.diag(e) > 0).all()


# ---------------------------------------------------------------- SCDM


def test_qrcp_pivots_match_lapack_geqp3():
    rng = np.random.default_rng(0)
    for trial in range(5):
        a = rng.standard_normal((6, 40))
        piv = O.qrcp_pivots(a, 6)
        _, _, p = scipy.linalg.qr(a, pivoting=True, mode="economic")
        assert list(piv) == list(p[:6])


def test_qrcp_pivot_ratios_flag_a_wrong_order():
    rng = np.random.default_rng(8)
    a = rng.standard_normal((5, 30))
    piv = O.qrcp_pivots(a, 5)
    assert np.allclose(O.qrcp_pivot_ratios(a, piv), 1.0)
    bad = list(piv)
    bad[1], bad[2] = bad[2], bad[1]
    assert O.qrcp_pivot_ratios(a, bad).min() < 0.999


def test_qrcp_tie_takes_lowest_index():
    a = np.zeros((2, 5))
    a[0, 3] = 1.0
    a[0, 1] = 1.0  # tie between columns 1 and 3
    a[1, 4] = 0.5
    piv = O.qrcp_pivots(a, 2)
    assert list(piv) == [1, 4]


def test_scdm_orthogonal_polar_and_localising():
    g, occ, _ = _small(seed=31, shape=(16, 16, 16), n_occ=8, n_centres=6, cell=(12.0, 12.0, 12.0))
    piv, u, w = O.scdm(g, occ, stride=2)
    assert len(set(piv.tolist())) == 8
    sub = set(O.subsample_indices(g.shape, 2).tolist())
    assert all(p in sub for p in piv.tolist())
    assert np.allclose(u.T @ u, np.eye(8), atol=1e-12)
    # U is the orthogonal polar factor of phi_C^T (independent route: SVD)
    phic = occ.reshape(8, -1)[:, piv].T
    uu, _, vt = np.linalg.svd(phic.T)
    assert np.allclose(u, uu @ vt, atol=1e-10)
    wm = w.reshape(8, -1)
    assert np.allclose(g.dv * wm @ wm.T, np.eye(8), atol=1e-12)
    # same span: projector unchanged
    om = occ.reshape(8, -1)
    c = g.dv * om @ wm.T
    assert np.allclose(c @ c.T, np.eye(8), atol=1e-12)
    # localisation reduces the off-diagonal overlap of moduli
    s0 = O.overlap_moduli(g, occ)
    s1 = O.overlap_moduli(g, w)
    off = ~np.eye(8, dtype=bool)
    assert s1[off].sum() < s0[off].sum()


def test_subsample_indices_odd_grid():
    idx = O.subsample_indices((5, 4, 3), 2)
    assert len(idx) == 3 * 2 * 2
    assert idx[0] == 0 and idx[1] == 2 and idx[2] == (0 * 4 + 2) * 3


# ---------------------------------------------------------------- screening


def test_alignment_recovers_a_rotated_set_and_is_optimal():
    g, occ, _ = _small(seed=21, n_occ=6)
    _, _, w = O.scdm(g, occ, 2)
    rng = np.random.default_rng(4)
    r = synth.random_orthogonal(6, rng)
    rotated = np.tensordot(r.T, w, axes=(1, 0))  # rotated_j = sum_i w_i r_ij
    q, aligned = O.align_orbitals(g, rotated, w)
    assert np.max(np.abs(aligned - w)) < 1e-12
    assert np.max(np.abs(q - r.T)) < 1e-12
    # a drifted set: the aligned one is orthonormal, spans the same space and is
    # closer to the reference than any other rotation tried
    drift = synth.small_localized_system(22, g.cell, g.shape, 6.0, 4, 6).phi
    new = O.lowdin(g, occ + 0.05 * drift)
    _, aligned = O.align_orbitals(g, new, w)
    a2 = aligned.reshape(6, -1)
    assert np.max(np.abs(g.dv * a2 @ a2.T - np.eye(6))) < 1e-12
    proj = g.dv * new.reshape(6, -1) @ a2.T
    assert np.max(np.abs(proj.T @ proj - np.eye(6))) < 1e-10  # same span
    dist = np.sum((aligned - w) ** 2)
    for _ in range(20):
        rr = synth.random_orthogonal(6, rng)
        other = np.tensordot(rr.T, aligned, axes=(1, 0))
        assert np.sum((other - w) ** 2) >= dist - 1e-12


def test_pw_basis_half_sphere_and_order():
    cell, ecut = (7.0, 8.0, 9.5), 6.0
    m = O.pw_basis(cell, ecut)
    g2 = np.sum((2 * np.pi * m / np.array(cell)) ** 2, axis=1)
    assert np.all(g2 / 2 < ecut) and np.all(np.diff(g2) >= 0) and tuple(m[0]) == (0, 0, 0)
    # every G of the full sphere is in the half sphere exactly once, as G or -G
    full = set()
    mm = [int(np.floor(np.sqrt(2 * ecut) * L / (2 * np.pi))) for L in cell]
    for m1 in range(-mm[0], mm[0] + 1):
        for m2 in range(-mm[1], mm[1] + 1):
            for m3 in range(-mm[2], mm[2] + 1):
                if (2 * np.pi * m1 / cell[0]) ** 2 + (2 * np.pi * m2 / cell[1]) ** 2 + (2 * np.pi * m3 / cell[2]) ** 2 < 2 * ecut:
                    full.add((m1, m2, m3))
    half = {tuple(x) for x in m}
    assert len(half) == len(m) and len(full) == 2 * len(m) - 1
    assert all((x in half) != ((-x[0], -x[1], -x[2]) in half) or x == (0, 0, 0) for x in full)


def test_pw_transforms_against_direct_sums():
    cell, shape, ecut = (7.0, 8.0, 9.5), (16, 18, 20), 6.0
    g = O.Grid(cell, shape)
    m = O.pw_basis(cell, ecut)
    rng = np.random.default_rng(9)
    coef = rng.standard_normal((2, len(m))) + 1j * rng.standard_normal((2, len(m)))
    phi = O.pw_to_grid(g, m, coef)
    gv = 2 * np.pi * m / np.array(cell)
    for (i, j, k) in ((0, 0, 0), (3, 11, 7), (15, 17, 19)):
        r = np.array([i * cell[0] / shape[0], j * cell[1] / shape[1], k * cell[2] / shape[2]])
        ph = np.exp(1j * gv @ r)
        direct = coef[:, 0].real + 2 * np.real(coef[:, 1:] @ ph[1:])
        assert np.max(np.abs(phi[:, i, j, k] - direct)) < 1e-11
    back = O.grid_to_pw(g, m, phi)
    assert np.max(np.abs(back[:, 1:] - coef[:, 1:])) < 1e-12
    assert np.max(np.abs(back[:, 0] - coef[:, 0].real)) < 1e-12
    # Parseval: dV sum phi^2 = Omega (c0^2 + 2 sum |c|^2)
    nrm = g.dv * np.sum(phi ** 2, axis=(1, 2, 3))
    assert np.allclose(nrm, g.omega * (coef[:, 0].real ** 2 + 2 * np.sum(np.abs(coef[:, 1:]) ** 2, axis=1)))


def test_overlap_moduli_diagonal_is_one_and_threshold_rule():
    g, occ, _ = _small(seed=41, n_occ=6)
    s = O.overlap_moduli(g, occ)
    assert np.allclose(np.diag(s), 1.0, atol=1e-12)
    thr = s[0, 1]
    keep = O.kept_pairs(s, thr, 6, 2)
    assert keep[0, 1] and keep[1, 0]  # S >= thr kept (drop only when S < thr)
    assert keep[:, 6:].all()  # pairs with extras always kept
    assert keep.shape == (6, 8)


def test_kept_count_monotone_and_zero_threshold_keeps_all():
    g, occ, _ = _small(seed=42, shape=(16, 16, 16), n_occ=8, n_centres=8, cell=(14.0, 14.0, 14.0))
    s = O.overlap_moduli(g, occ)
    counts = [O.kept_pairs(s, t, 8, 0).sum() for t in (0.0, 1e-4, 1e-3, 1e-2, 0.1, 0.5)]
    assert counts[0] == 64
    assert all(a >= b for a, b in zip(counts, counts[1:]))


# ---------------------------------------------------------------- ACE


def test_ace_exact_on_building_set_and_its_span():
    g, occ, extra = _small(seed=51, n_occ=5, n_extra=2)
    keep = np.ones((5, 7), dtype=bool)
    W, _, _ = O.apply_exchange(g, occ, extra, keep)
    psi = np.concatenate([occ, extra])
    xi, l, m = O.ace_build(g, psi, W, "avg")
    kace = O.ace_apply(g, xi, psi)
    assert np.max(np.abs(kace - W)) <= 1e-12 * np.max(np.abs(W))
    c = np.random.default_rng(2).standard_normal((3, 7))
    comb = np.tensordot(c, psi, axes=(1, 0))
    kc = np.tensordot(c, W, axes=(1, 0))
    assert np.max(np.abs(O.ace_apply(g, xi, comb) - kc)) <= 1e-12 * np.max(np.abs(kc))
    # Cholesky factor: -M = L L^T, L lower triangular with positive diagonal
    assert np.allclose(l @ l.T, -m, atol=1e-13 * np.abs(m).max())
    assert (np.diag(l) > 0).all() and np.allclose(l, np.tril(l))


def test_ace_inner_projection_bound():
    g, occ, _ = _small(seed=52, n_occ=5)
    keep = np.ones((5, 5), dtype=bool)
    W, _, _ = O.apply_exchange(g, occ, None, keep)
    xi, _, _ = O.ace_build(g, occ, W)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((4,) + g.shape)
    kpsi, _ = O.apply_exchange_columns(g, occ, psi, np.ones((5, 4), dtype=bool))
    kace = O.ace_apply(g, xi, psi)
    for t in range(4):
        ek = g.dv * np.sum(psi[t] * kpsi[t])
        ea = g.dv * np.sum(psi[t] * kace[t])
        assert ek <= ea + 1e-12 * abs(ek)
        assert ea <= 1e-14


def test_lace_zero_threshold_equals_ace():
    g, occ, _ = _small(seed=53, n_occ=5)
    s = O.overlap_moduli(g, occ)
    keep0 = O.kept_pairs(s, 0.0, 5, 0)
    W0, ex0, _ = O.apply_exchange(g, occ, None, keep0)
    W1, ex1, _ = O.apply_exchange(g, occ, None, np.ones((5, 5), dtype=bool))
    assert np.array_equal(W0, W1) and ex0 == ex1


def test_symmetrization_modes():
    m = np.arange(9.0).reshape(3, 3)
    assert np.allclose(O.symmetrize(m, "avg"), (m + m.T) / 2)
    up = O.symmetrize(m, "upper")
    assert np.allclose(up, up.T) and up[2, 0] == m[0, 2]
    lo = O.symmetrize(m, "lower")
    assert np.allclose(lo, lo.T) and lo[0, 2] == m[2, 0]


def test_truncated_exchange_matrix_stays_negative_definite():
    # Sec. 2: M' should stay invertible for small truncations
    g, occ, _ = _small(seed=54, shape=(16, 16, 16), n_occ=8, n_centres=8, cell=(14.0, 14.0, 14.0))
    _, _, w = O.scdm(g, occ)
    s = O.overlap_moduli(g, w)
    keep = O.kept_pairs(s, 5e-3, 8, 0)
    W, _, _ = O.apply_exchange(g, w, None, keep)
    xi, l, m = O.ace_build(g, w, W, "avg")
    assert np.linalg.eigvalsh(m).max() < 0


# ---------------------------------------------------------------- planted mistakes


def test_planted_kernel_mistake_is_caught(monkeypatch):
    """A kernel without the 4 pi factor must fail the closed-form pin."""
    good = O.lace_oracle.coulomb_kernel
    monkeypatch.setattr(O.lace_oracle, "coulomb_kernel", lambda grid: good(grid) / (4 * np.pi))
    a, L, n = 1.0, 10.0, 32
    phi = _periodic_gaussian_orbital(a, L, n, centre=(5.0, 5.0, 5.0))[None]
    g = O.Grid((L, L, L), (n, n, n))
    _, ex, _ = O.apply_exchange(g, phi, None, np.ones((1, 1), dtype=bool))
    closed = np.sqrt(2 * a / np.pi) - 2.8372974794806 / L + 2 * np.pi / (a * L ** 3)
    assert abs(ex + 0.5 * closed) > 1e-3


def test_planted_transpose_mistake_is_caught(monkeypatch):
    """Applying U^T instead of U in SCDM breaks the polar-factor pin."""
    g, occ, _ = _small(seed=31, shape=(16, 16, 16), n_occ=8, n_centres=6, cell=(12.0, 12.0, 12.0))
    piv, u, w = O.scdm(g, occ)
    w_bad = np.tensordot(u, occ, axes=(1, 0))  # sum_k U_mk phi_k (transposed)
    s_good = O.overlap_moduli(g, w)
    s_bad = O.overlap_moduli(g, w_bad)
    assert not np.allclose(s_good, s_bad, atol=1e-6)
