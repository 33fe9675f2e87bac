"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP64 path must match E_x to |dE_x| <= 1e-6 Ha and the mixed
(FP32 FFT) path to |dE_x| <= 1e-5 Ha per orbital set; orbitals and W are
compared element by element with a relative bound derived from the
arithmetic (FP64: a few hundred ulps of the largest element; FP32: the
accumulated rounding of an FFT of length Ng, ~1e-6 of the largest element).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_FP64, LACE_MIXED, Lace, LaceError
from paper_1801_09263_gb300 import binding as B

pytestmark = pytest.mark.gpu

EX_TOL = {LACE_FP64: 1e-6, LACE_MIXED: 1e-5}
REL_TOL = {LACE_FP64: 1e-10, LACE_MIXED: 2e-5}
PRECS = [LACE_FP64, LACE_MIXED]
PNAME = {LACE_FP64: "fp64", LACE_MIXED: "mixed"}


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_ctx(sysm, prec, ortho=True):
    ctx = Lace(0, prec)
    ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
    ctx.load_orbitals(sysm.phi, sysm.n_occ, sysm.n_extra, ortho)
    return ctx


def oracle_orbitals(sysm):
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi[: sysm.n_occ])
    extra = O.orthonormalize_extras(g, occ, sysm.phi[sysm.n_occ:]) if sysm.n_extra else None
    return g, occ, extra


def keep_from_pairs(pairs, n_occ, n_extra):
    keep = np.zeros((n_occ, n_occ + n_extra), dtype=bool)
    for i, j in pairs:
        keep[i, j] = True
        if j < n_occ:
            keep[j, i] = True
    return keep


@pytest.fixture(scope="module")
def cfg1():
    return synth.config1_plain()


@pytest.fixture(scope="module")
def cfg1_ref(cfg1):
    g, occ, _ = oracle_orbitals(cfg1)
    W, ex, e = O.apply_exchange(g, occ, None, np.ones((8, 8), dtype=bool))
    return occ, W, ex


@pytest.fixture(scope="module")
def small_loc():
    # 36^3 grid (radix 4 x 9), 20 occupied orbitals on 14 centres, 4 extras
    return synth.small_localized_system(77, (13.0, 13.0, 13.0), (36, 36, 36), 12.0, 14, 20, 4)


# ------------------------------------------------------------------ plain exchange (configuration 1)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_plain_exchange_24cubed_8_orbitals(cfg1, cfg1_ref, prec):
    occ, W_ref, ex_ref = cfg1_ref
    with make_ctx(cfg1, prec) as ctx:
        psi = ctx.get_orbitals(B.ORB_PSI)
        assert relerr(psi, occ) < REL_TOL[prec]
        W, ex = ctx.apply_exchange()
        assert abs(ex - ex_ref) <= EX_TOL[prec], (ex, ex_ref)
        assert relerr(W, W_ref) < REL_TOL[prec]
        assert ctx.exchange_energy(2.0) == pytest.approx(2 * ex, rel=1e-15)
        # pair energies: e_ij = (ij|ji), symmetric, positive diagonal
        e = ctx.get_matrix(B.MAT_PAIR_ENERGY)
        assert np.allclose(e, e.T) and (np.diag(e) > 0).all()
        assert abs(-0.5 * e.sum() - ex) <= 1e-12 * abs(ex)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_overlap_of_moduli_with_partial_tiles(prec):
    """150 orbitals: two 128-row tiles of the tensor-core Gram (the second
    partial), the three symmetric tiles only, against the oracle's Eq. 4 on
    the oracle's SCDM orbitals at the same pivots."""
    sysm = synth.small_localized_system(93, (13.0, 13.0, 13.0), (36, 36, 36), 12.0, 120, 150, 0)
    g, occ, _ = oracle_orbitals(sysm)
    piv, _, w = O.scdm(g, occ, 2)
    s_ref = O.overlap_moduli(g, w)
    with make_ctx(sysm, prec) as ctx:
        ctx.set_pivots(piv)
        n = ctx.screen(1e-3)
        s = ctx.get_matrix(B.MAT_OVERLAP_MODULI)
        pairs = ctx.get_pairs()
    assert relerr(s, s_ref) < (1e-10 if prec == LACE_FP64 else 1e-5)
    keep = keep_from_pairs(pairs, 150, 0)
    keep_ref = O.kept_pairs(s_ref, 1e-3, 150, 0)
    band = np.abs(s_ref - 1e-3) <= 1e-4 * 1e-3
    assert not ((keep != keep_ref) & ~band).any()
    assert n == len(pairs) == int(np.triu(keep).sum())


@pytest.mark.parametrize("n_occ,centres", [(100, 80), (300, 120)])
def test_host_load_matches_the_device_load(n_occ, centres):
    """Mixed precision, 100 and 300 orbitals (2 and 5 tiles of the Loewdin
    overlap, the last one partial): orbitals loaded from host arrays are
    bit-identical to those of lace_load_orbitals_dev, and close to the
    oracle's symmetric orthonormalisation (overlap condition numbers ~200
    and ~1,000 here)."""
    torch = pytest.importorskip("torch")
    sysm = synth.small_localized_system(91, (13.0, 13.0, 13.0), (36, 36, 36), 12.0, centres, n_occ, 0)
    with make_ctx(sysm, LACE_MIXED) as ctx:
        psi_host = ctx.get_orbitals(B.ORB_PSI)
    with Lace(0, LACE_MIXED) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals_dev(torch.from_numpy(sysm.phi).cuda(), n_occ, 0, True)
        psi_dev = ctx.get_orbitals(B.ORB_PSI)
    assert np.array_equal(psi_host, psi_dev)
    occ = O.lowdin(O.Grid(sysm.cell, sysm.shape), sysm.phi)
    assert relerr(psi_host, occ) < 1e-4


@pytest.mark.parametrize("shape,cell", [((45, 45, 45), (11.0, 11.0, 11.0)),
                                        ((24, 30, 20), (9.0, 11.0, 8.0)),
                                        ((25, 27, 32), (9.5, 10.0, 12.0))])
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_plain_exchange_odd_and_noncubic_grids(shape, cell, prec):
    sysm = synth.small_localized_system(5, cell, shape, 6.0, 3, 5, mix=True)
    g, occ, _ = oracle_orbitals(sysm)
    W_ref, ex_ref, _ = O.apply_exchange(g, occ, None, np.ones((5, 5), dtype=bool))
    with make_ctx(sysm, prec) as ctx:
        W, ex = ctx.apply_exchange()
    assert abs(ex - ex_ref) <= EX_TOL[prec]
    assert relerr(W, W_ref) < REL_TOL[prec]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_single_orbital_and_odd_pair_count(prec):
    # 1 orbital -> 1 pair (one complex grid with an empty second slot)
    sysm = synth.small_localized_system(9, (8.0, 8.0, 8.0), (16, 16, 16), 5.0, 1, 1)
    g, occ, _ = oracle_orbitals(sysm)
    W_ref, ex_ref, _ = O.apply_exchange(g, occ, None, np.ones((1, 1), dtype=bool))
    with make_ctx(sysm, prec) as ctx:
        W, ex = ctx.apply_exchange()
        assert len(ctx.get_pairs()) == 1
    assert abs(ex - ex_ref) <= EX_TOL[prec]
    assert relerr(W, W_ref) < REL_TOL[prec]


# Every cubic size with compile-time specialised FP32 passes: the
# out-of-place passes (24 ... 100) and the in-place ones (128, whose two planes
# do not fit on chip).  3 occupied + 1 extra orbital: 6 occupied pairs and 3
# occupied-extra pairs, 5 complex grids of which the last holds one pair.
SPEC_SIZES = [24, 32, 36, 40, 48, 50, 54, 60, 64, 72, 80, 96, 100, 128]


@pytest.mark.parametrize("n", SPEC_SIZES)
def test_size_specialised_fft_passes_match_oracle(n):
    side = 10.0 * n / 48
    sysm = synth.small_localized_system(400 + n, (side, side, side), (n, n, n), 10.0, 3, 3, 1)
    g, occ, extra = oracle_orbitals(sysm)
    W_ref, ex_ref, _ = O.apply_exchange(g, occ, extra, np.ones((3, 4), dtype=bool))
    with make_ctx(sysm, LACE_MIXED) as ctx:
        W, ex = ctx.apply_exchange()
        assert len(ctx.get_pairs()) == 9
    assert abs(ex - ex_ref) <= EX_TOL[LACE_MIXED], (ex, ex_ref)
    assert relerr(W, W_ref) < REL_TOL[LACE_MIXED]


# ------------------------------------------------------------------ SCDM, screening, L-ACE


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_scdm_pivots_are_a_valid_qrcp_order(small_loc, prec):
    g, occ, _ = oracle_orbitals(small_loc)
    with make_ctx(small_loc, prec) as ctx:
        piv = ctx.localize(2)
    sub = O.subsample_indices(g.shape, 2)
    pos = {int(v): k for k, v in enumerate(sub)}
    assert all(int(p) in pos for p in piv)
    cols = [pos[int(p)] for p in piv]
    ratios = O.qrcp_pivot_ratios(occ.reshape(small_loc.n_occ, -1)[:, sub], cols)
    tol = 1e-9 if prec == LACE_FP64 else 1e-4
    assert ratios.min() >= 1 - tol, ratios.min()
    ref = O.qrcp_pivots(occ.reshape(small_loc.n_occ, -1)[:, sub], small_loc.n_occ)
    if prec == LACE_FP64:
        assert list(sub[ref]) == [int(p) for p in piv]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_scdm_pivots_are_deterministic(prec):
    # the persistent QR runs on every SM with a grid barrier per step; repeated
    # runs (and a second context) must select the same pivots
    # 200 rows x 46,656 columns: tiles in registers and in shared memory
    sysm = synth.small_localized_system(13, (23.5, 23.5, 23.5), (72, 72, 72), 40.0, 150, 200)
    out = []
    for _ in range(2):
        with make_ctx(sysm, prec) as ctx:
            out.append([ctx.localize(2) for _ in range(2)])
    ref = out[0][0]
    assert all((p == ref).all() for run in out for p in run)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_alignment_to_previous_orbitals_matches_oracle(small_loc, prec):
    g, occ1, _ = oracle_orbitals(small_loc)
    n = small_loc.n_occ
    drift = synth.small_localized_system(78, small_loc.cell, small_loc.shape, small_loc.ecut, 14, n).phi
    phi2 = small_loc.phi.copy()
    phi2[:n] += 0.05 * drift
    with make_ctx(small_loc, prec) as ctx:
        piv1 = ctx.localize(2)
        assert ctx.align_to_previous() is False  # first call: reference only
        ctx.load_orbitals(phi2, n, small_loc.n_extra, True)
        piv2 = ctx.localize(2)
        assert ctx.align_to_previous() is True
        psi2 = ctx.get_orbitals(B.ORB_PSI)[:n]
        u = ctx.get_matrix(B.MAT_SCDM_U)
    _, _, w1 = O.scdm(g, occ1, 2, pivots=piv1)
    occ2 = O.lowdin(g, phi2[:n])
    _, u2, w2 = O.scdm(g, occ2, 2, pivots=piv2)
    q, aligned = O.align_orbitals(g, w2, w1)
    tol = 1e-10 if prec == LACE_FP64 else 2e-5
    assert relerr(psi2, aligned) < tol
    assert relerr(u, u2 @ q) < (1e-10 if prec == LACE_FP64 else 1e-5)
    # closer to the previous set than the unaligned localised orbitals
    assert np.sum((psi2 - w1) ** 2) <= np.sum((w2 - w1) ** 2) + 1e-12


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_scdm_rotation_with_imposed_pivots(small_loc, prec):
    g, occ, _ = oracle_orbitals(small_loc)
    piv, u_ref, w_ref = O.scdm(g, occ, 2)
    with make_ctx(small_loc, prec) as ctx:
        ctx.set_pivots(piv)
        u = ctx.get_matrix(B.MAT_SCDM_U)
        psi = ctx.get_orbitals(B.ORB_PSI)
    assert relerr(u, u_ref) < (1e-9 if prec == LACE_FP64 else 1e-4)
    assert relerr(psi[: small_loc.n_occ], w_ref) < (1e-9 if prec == LACE_FP64 else 1e-4)


@pytest.mark.parametrize("thr", [0.0, 1e-3, 2e-2])
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_screened_exchange_matches_oracle(small_loc, prec, thr):
    g, occ, extra = oracle_orbitals(small_loc)
    n, ne = small_loc.n_occ, small_loc.n_extra
    piv, _, w = O.scdm(g, occ, 2)
    s_ref = O.overlap_moduli(g, w)
    with make_ctx(small_loc, prec) as ctx:
        ctx.set_pivots(piv)
        npairs = ctx.screen(thr)
        s = ctx.get_matrix(B.MAT_OVERLAP_MODULI)
        pairs = ctx.get_pairs()
        W, ex = ctx.apply_exchange()
    assert relerr(s, s_ref) < (1e-10 if prec == LACE_FP64 else 1e-5)
    keep_gpu = keep_from_pairs(pairs, n, ne)
    keep_ref = O.kept_pairs(s_ref, thr, n, ne)
    band = np.abs(s_ref - thr) <= 1e-5 * max(thr, 1e-300)
    differ = keep_gpu[:, :n] != keep_ref[:, :n]
    assert not (differ & ~band).any()
    assert (keep_gpu[:, n:]).all()
    assert npairs == len(pairs) == int(np.triu(keep_gpu[:, :n]).sum()) + n * ne
    # parity on the GPU's kept set (identical to the oracle's outside the tie band)
    W_ref, ex_ref, _ = O.apply_exchange(g, w, extra, keep_gpu)
    assert abs(ex - ex_ref) <= EX_TOL[prec], (ex, ex_ref)
    assert relerr(W, W_ref) < REL_TOL[prec]


# ------------------------------------------------------------------ ACE


@pytest.mark.parametrize("sym", [B.LACE_SYM_AVG, B.LACE_SYM_UPPER, B.LACE_SYM_LOWER])
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_ace_build_and_apply(small_loc, prec, sym):
    g, occ, extra = oracle_orbitals(small_loc)
    n, ne = small_loc.n_occ, small_loc.n_extra
    piv, _, w = O.scdm(g, occ, 2)
    rng = np.random.default_rng(3)
    probe = rng.standard_normal((3,) + g.shape)
    with make_ctx(small_loc, prec) as ctx:
        ctx.set_pivots(piv)
        ctx.screen(1e-3)
        pairs = ctx.get_pairs()
        W, _ = ctx.apply_exchange()
        ctx.build_ace(sym)
        m = ctx.get_matrix(B.MAT_EXCHANGE)
        l = ctx.get_matrix(B.MAT_CHOLESKY)
        xi = ctx.get_orbitals(B.ORB_XI)
        psi = ctx.get_orbitals(B.ORB_PSI)
        k_on_psi = ctx.apply_ace(psi)
        k_probe = ctx.apply_ace(probe)
        e_probe = ctx.ace_energy()  # the host apply runs in chunks (mixed path): their energies summed
    keep = keep_from_pairs(pairs, n, ne)
    W_ref, _, _ = O.apply_exchange(g, w, extra, keep)
    psi_ref = np.concatenate([w, extra])
    mode = {B.LACE_SYM_AVG: "avg", B.LACE_SYM_UPPER: "upper", B.LACE_SYM_LOWER: "lower"}[sym]
    xi_ref, l_ref, m_ref = O.ace_build(g, psi_ref, W_ref, mode)
    tol = 1e-9 if prec == LACE_FP64 else 5e-5
    assert relerr(m, g.dv * psi_ref.reshape(n + ne, -1) @ W_ref.reshape(n + ne, -1).T) < tol
    assert relerr(l, l_ref) < tol
    assert relerr(xi, xi_ref) < tol
    # with truncation M' is not symmetric, so ACE is not exact on Psi: compare with the oracle's K_ACE
    assert relerr(k_on_psi, O.ace_apply(g, xi_ref, psi_ref)) < tol
    assert relerr(k_probe, O.ace_apply(g, xi_ref, probe)) < tol
    # the block ACE energy sum_j <probe_j|K_ACE|probe_j> of the last application
    e_ref = g.dv * float(np.sum(probe * O.ace_apply(g, xi_ref, probe)))
    assert abs(e_probe - e_ref) <= tol * abs(e_ref), (e_probe, e_ref)


def test_host_ace_apply_in_uneven_chunks(small_loc):
    """Mixed precision, 5 host functions: the chunked host apply runs chunks
    of 2, 2 and 1 functions and an empty fourth; its result is bit-identical
    to the device apply of the same functions (the same tiles and K chunks),
    and the chunk energies sum to the device apply's block energy."""
    torch = pytest.importorskip("torch")
    g, occ, _ = oracle_orbitals(small_loc)
    piv, _, _ = O.scdm(g, occ, 2)
    probe = np.random.default_rng(11).standard_normal((5,) + g.shape)
    with make_ctx(small_loc, LACE_MIXED) as ctx:
        ctx.set_pivots(piv)
        ctx.screen(1e-3)
        ctx.apply_exchange()
        ctx.build_ace()
        k_host = ctx.apply_ace(probe)
        e_host = ctx.ace_energy()
        p_dev = torch.from_numpy(probe).cuda()
        k_dev = torch.empty_like(p_dev)
        ctx.apply_ace_dev(p_dev, k_dev)
        e_dev = ctx.ace_energy()
    assert np.array_equal(k_host, k_dev.cpu().numpy())
    assert abs(e_host - e_dev) <= 1e-12 * abs(e_dev)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_ace_on_a_grid_with_an_odd_point_count(prec):
    # 25 x 27 x 45 points: rows of the orbital arrays are not 16-byte aligned
    sysm = synth.small_localized_system(41, (9.5, 10.0, 16.0), (25, 27, 45), 6.0, 6, 8, 3)
    g, occ, extra = oracle_orbitals(sysm)
    probe = np.random.default_rng(5).standard_normal((2,) + g.shape)
    with make_ctx(sysm, prec) as ctx:
        piv = ctx.localize(2)
        ctx.screen(0.0)
        W, ex = ctx.apply_exchange()
        ctx.build_ace()
        k_probe = ctx.apply_ace(probe)
    _, _, w = O.scdm(g, occ, 2, pivots=piv)
    W_ref, ex_ref, _ = O.apply_exchange(g, w, extra, np.ones((8, 11), dtype=bool))
    xi_ref, _, _ = O.ace_build(g, np.concatenate([w, extra]), W_ref)
    tol = 1e-9 if prec == LACE_FP64 else 5e-5
    assert abs(ex - ex_ref) <= EX_TOL[prec]
    assert relerr(k_probe, O.ace_apply(g, xi_ref, probe)) < tol


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_screened_kernel_exchange_and_ace_match_oracle(small_loc, prec):
    # erfc-screened short-range kernel (range-separated hybrids, Sec. 4) with the
    # exchange fraction 0.25; L-ACE on the oracle's pivots
    w, alpha = 0.4, 0.25
    g0, occ, extra = oracle_orbitals(small_loc)
    g = O.Grid(g0.cell, g0.shape, kernel="erfc", screening=w, alpha=alpha)
    n, ne = small_loc.n_occ, small_loc.n_extra
    piv, _, wl = O.scdm(g, occ, 2)
    probe = np.random.default_rng(8).standard_normal((2,) + g.shape)
    with make_ctx(small_loc, prec) as ctx:
        ctx.set_kernel(B.KERNEL_ERFC, w, alpha)
        ctx.set_pivots(piv)
        ctx.screen(1e-3)
        keep = keep_from_pairs(ctx.get_pairs(), n, ne)
        W, ex = ctx.apply_exchange()
        ctx.build_ace()
        k_probe = ctx.apply_ace(probe)
    W_ref, ex_ref, _ = O.apply_exchange(g, wl, extra, keep)
    assert abs(ex - ex_ref) <= EX_TOL[prec]
    assert relerr(W, W_ref) < REL_TOL[prec]
    xi_ref, _, _ = O.ace_build(g, np.concatenate([wl, extra]), W_ref)
    assert relerr(k_probe, O.ace_apply(g, xi_ref, probe)) < (1e-9 if prec == LACE_FP64 else 5e-5)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_ace_exact_on_building_set_without_truncation(small_loc, prec):
    # Sec. 2: ACE equals the exchange operator on the functions used to build it
    with make_ctx(small_loc, prec) as ctx:
        ctx.localize(2)
        ctx.screen(0.0)
        W, _ = ctx.apply_exchange()
        ctx.build_ace()
        psi = ctx.get_orbitals(B.ORB_PSI)
        k_on_psi = ctx.apply_ace(psi)
        comb = np.tensordot(np.random.default_rng(1).standard_normal((2, psi.shape[0])), psi, axes=(1, 0))
        k_comb = ctx.apply_ace(comb)
    assert relerr(k_on_psi, W) < (1e-9 if prec == LACE_FP64 else 1e-4)
    w_comb = np.tensordot(np.random.default_rng(1).standard_normal((2, psi.shape[0])), W, axes=(1, 0))
    assert relerr(k_comb, w_comb) < (1e-9 if prec == LACE_FP64 else 1e-4)


# ------------------------------------------------------------------ edge cases and errors


def test_threshold_above_one_drops_every_pair():
    sysm = synth.small_localized_system(12, (8.0, 8.0, 8.0), (16, 16, 16), 5.0, 3, 3)
    with make_ctx(sysm, LACE_FP64) as ctx:
        assert ctx.screen(2.0) == 0
        W, ex = ctx.apply_exchange()
    assert ex == 0.0 and not W.any()


def test_out_of_order_calls_and_bad_sizes():
    ctx = Lace(0, LACE_FP64)
    with pytest.raises(LaceError) as e:
        ctx.apply_exchange()
    assert e.value.status == 2
    with pytest.raises(LaceError) as e:
        ctx.set_cell((10.0, 10.0, 10.0), (7, 8, 8), 5.0)
    assert e.value.status == 7
    ctx.set_cell((10.0, 10.0, 10.0), (16, 16, 16), 5.0)
    sysm = synth.small_localized_system(13, (10.0, 10.0, 10.0), (16, 16, 16), 5.0, 2, 2)
    ctx.load_orbitals(sysm.phi, 2, 0)
    with pytest.raises(LaceError) as e:
        ctx.build_ace()
    assert e.value.status == 2
    with pytest.raises(LaceError) as e:
        ctx.set_pivots([0, 0])
    assert e.value.status == 1
    ctx.close()


def test_linearly_dependent_orbitals_are_rejected():
    sysm = synth.small_localized_system(14, (10.0, 10.0, 10.0), (16, 16, 16), 5.0, 2, 2)
    phi = np.concatenate([sysm.phi, sysm.phi[:1]])
    ctx = Lace(0, LACE_FP64)
    ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
    with pytest.raises(LaceError) as e:
        ctx.load_orbitals(phi, 3, 0, True)
    assert e.value.status == 5
    ctx.close()


# ------------------------------------------------------------------ size-specialised FP32 kernels


@pytest.mark.parametrize("n", [48, 64, 72, 96, 128])
def test_specialised_sizes_match_oracle(n):
    # cubic grids with n % 4 == 0 run the compile-time-specialised passes in FP32
    sysm = synth.small_localized_system(21 + n, (12.0, 12.0, 12.0), (n, n, n), 10.0, 3, 3)
    g, occ, _ = oracle_orbitals(sysm)
    W_ref, ex_ref, _ = O.apply_exchange(g, occ, None, np.ones((3, 3), dtype=bool))
    with make_ctx(sysm, LACE_MIXED) as ctx:
        W, ex = ctx.apply_exchange()
    assert abs(ex - ex_ref) <= EX_TOL[LACE_MIXED]
    assert relerr(W, W_ref) < REL_TOL[LACE_MIXED]


def test_specialised_and_generic_fp32_passes_agree(small_loc, monkeypatch):
    with make_ctx(small_loc, LACE_MIXED) as ctx:
        ctx.localize(2)
        ctx.screen(1e-3)
        W_spec, ex_spec = ctx.apply_exchange()
        monkeypatch.setenv("LACE_GENERIC_FFT", "1")
        W_gen, ex_gen = ctx.apply_exchange()
    assert abs(ex_spec - ex_gen) <= 1e-6
    assert relerr(W_spec, W_gen) < 1e-5


def test_tensor_core_ace_contraction_matches_fp32_cuda_cores(small_loc, monkeypatch):
    # mixed path: M = dV Psi^T W on tcgen05 (3xBF16 products, FP32 accumulate) vs the FP32 CUDA-core kernel
    mats = {}
    for notc in ("0", "1"):
        monkeypatch.setenv("LACE_NO_TC", notc)
        with make_ctx(small_loc, LACE_MIXED) as ctx:
            ctx.localize(2)
            ctx.screen(1e-3)
            ctx.apply_exchange(want_W=False)
            ctx.build_ace()
            probe = np.random.default_rng(4).standard_normal((2,) + small_loc.shape)
            mats[notc] = (ctx.get_matrix(B.MAT_EXCHANGE), ctx.apply_ace(probe))
    m_tc, k_tc = mats["0"]
    m_cc, k_cc = mats["1"]
    assert relerr(m_tc, m_cc) < 2e-5
    assert relerr(k_tc, k_cc) < 5e-5
