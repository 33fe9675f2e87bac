"""Full-size ACE workload: 96^3 grid, 256 water-like occupied + 128 extra orbitals.

L-ACE at S_thr = 1e-3 on the mixed path (tensor-core ACE contractions).  The
oracle checks E_x over the GPU's kept pairs and the exchange on sampled
targets (occupied and extra); the ACE factors are checked against their
definitions with the GPU's own M and W: -M'_sym = L L^T, xi = W L^{-T} on
sampled columns, K_ACE psi = -xi (dV xi^T psi) on a probe.
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_MIXED, Lace
from paper_1801_09263_gb300 import binding as B

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def run():
    sysm = synth.config3_water_like_with_extras()
    probe = np.random.default_rng(7).standard_normal((2,) + sysm.shape)
    with Lace(0, LACE_MIXED) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, 256, 128, True)
        piv = ctx.localize(2)
        ctx.screen(1e-3)
        W, ex = ctx.apply_exchange()
        ctx.build_ace()
        out = dict(piv=piv, W=W, ex=ex, pairs=ctx.get_pairs(), psi=ctx.get_orbitals(B.ORB_PSI),
                   M=ctx.get_matrix(B.MAT_EXCHANGE), L=ctx.get_matrix(B.MAT_CHOLESKY),
                   xi=ctx.get_orbitals(B.ORB_XI), probe=probe, kprobe=ctx.apply_ace(probe))
    return sysm, out


def test_energy_and_sampled_columns_match_oracle(run):
    sysm, r = run
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi[:256])
    extra = O.orthonormalize_extras(g, occ, sysm.phi[256:])
    _, _, w = O.scdm(g, occ, 2, pivots=r["piv"])
    keep = np.zeros((256, 384), dtype=bool)
    for i, j in r["pairs"]:
        keep[i, j] = True
        if j < 256:
            keep[j, i] = True
    assert keep[:, 256:].all()
    e = 0.0
    for j in range(256):
        ii = np.nonzero(keep[: j + 1, j])[0]
        rho = w[ii] * w[j][None]
        v = O.pair_potential(g, rho)
        eij = g.dv * np.sum((rho * v).reshape(len(ii), -1), axis=1)
        e += np.sum(np.where(ii == j, 1.0, 2.0) * eij)
    assert abs(r["ex"] - (-0.5 * e)) <= 1e-5
    psi = np.concatenate([w, extra])
    for j in (3, 200, 256, 383):
        Wj, _ = O.apply_exchange_columns(g, w, psi[j:j + 1], keep[:, j:j + 1])
        assert np.max(np.abs(r["W"][j] - Wj[0])) <= 2e-5 * np.max(np.abs(Wj[0]))


def test_ace_factors_match_their_definitions(run):
    sysm, r = run
    g = O.Grid(sysm.cell, sysm.shape)
    n = 384
    m_sym = 0.5 * (r["M"] + r["M"].T)
    L = r["L"]
    assert np.allclose(L, np.tril(L)) and (np.diag(L) > 0).all()
    assert np.max(np.abs(L @ L.T + m_sym)) <= 1e-12 * np.max(np.abs(m_sym))
    # M' = dV Psi^T W (tensor cores, 3xBF16) against FP64 products of the GPU's own Psi and W
    P = r["psi"].reshape(n, -1)
    Wm = r["W"].reshape(n, -1)
    for j in (0, 255, 300):
        mj = g.dv * P @ Wm[j]
        assert np.max(np.abs(r["M"][:, j] - mj)) <= 5e-5 * np.max(np.abs(mj))
    # xi = W L^{-T} on sampled columns
    Linv = np.linalg.inv(L)
    for k in (0, 100, 383):
        xk = (Linv[k] @ Wm)
        assert np.max(np.abs(r["xi"][k].ravel() - xk)) <= 5e-5 * np.max(np.abs(xk))
    # K_ACE probe
    X = r["xi"].reshape(n, -1)
    f = r["probe"].reshape(2, -1)
    c = g.dv * X @ f.T
    kref = -(c.T @ X)
    assert np.max(np.abs(r["kprobe"].reshape(2, -1) - kref)) <= 5e-5 * np.max(np.abs(kref))
