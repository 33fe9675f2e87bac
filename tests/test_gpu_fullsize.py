"""Full-size parity on the benchmark workload (72^3 grid, 256 water-like orbitals).

The step runs exactly as bench.py times it (Loewdin, SCDM on the 1/8
subsample, S_thr = 1e-3, pair convolutions).  The oracle checks what it can
compute at this size: E_x over the GPU's kept pairs (with the GPU's pivots)
and the exchange on a sample of target orbitals, one by one.
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_FP64, LACE_MIXED, Lace
from paper_1801_09263_gb300 import binding as B

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def runs():
    sysm = synth.config2_water_like()
    out = {}
    for prec in (LACE_FP64, LACE_MIXED):
        with Lace(0, prec) as ctx:
            ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
            ctx.load_orbitals(sysm.phi, 256, 0, True)
            piv = ctx.localize(2)
            n = ctx.screen(1e-3)
            W, ex = ctx.apply_exchange()
            out[prec] = dict(piv=piv, n=n, W=W, ex=ex, pairs=ctx.get_pairs(), psi=ctx.get_orbitals(B.ORB_PSI))
    return sysm, out


def test_mixed_matches_fp64_energy_at_full_size(runs):
    _, out = runs
    assert abs(out[LACE_MIXED]["ex"] - out[LACE_FP64]["ex"]) <= 1e-5


def test_fp64_energy_and_sampled_columns_match_oracle(runs):
    sysm, out = runs
    r = out[LACE_FP64]
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi)
    _, _, w = O.scdm(g, occ, 2, pivots=r["piv"])
    assert np.max(np.abs(r["psi"] - w)) <= 1e-9 * np.max(np.abs(w))
    keep = np.zeros((256, 256), dtype=bool)
    for i, j in r["pairs"]:
        keep[i, j] = keep[j, i] = True
    # E_x from the oracle's pair integrals over the kept set (each unordered pair once)
    e = 0.0
    for j in range(256):
        ii = np.nonzero(keep[: j + 1, j])[0]
        rho = w[ii] * w[j][None]
        v = O.pair_potential(g, rho)
        eij = g.dv * np.sum((rho * v).reshape(len(ii), -1), axis=1)
        e += np.sum(np.where(ii == j, 1.0, 2.0) * eij)
    ex_ref = -0.5 * e
    assert abs(r["ex"] - ex_ref) <= 1e-6, (r["ex"], ex_ref)
    # sampled targets: K psi_j one by one
    for j in (0, 77, 128, 255):
        Wj, _ = O.apply_exchange_columns(g, w, w[j:j + 1], keep[:, j:j + 1])
        assert np.max(np.abs(r["W"][j] - Wj[0])) <= 1e-10 * np.max(np.abs(Wj[0]))
        Wm = out[LACE_MIXED]["W"][j]
        assert np.max(np.abs(Wm - Wj[0])) <= 2e-5 * np.max(np.abs(Wj[0]))
