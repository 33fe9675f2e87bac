"""Accuracy of the tensor-core Grams on the benchmark workload (72^3, 256 orbitals).

The mixed path forms the overlap of moduli (Eq. 4) and the ACE matrix
M' = dV Psi^T W (Eq. 3) with tcgen05 MMAs on BF16 hi/lo splits.  The tensor
cores' FP32 accumulation is biased over long sums, so the kernel accumulates
a few K steps per TMEM accumulator and adds the period sums in compensated
FP32; these tests bound what is left:

* S against the oracle's overlap of moduli of the oracle's SCDM orbitals (at
  the GPU's pivots): diagonal bias, the error of the entries around S_thr,
  and the kept pairs;
* M' against the same contraction on CUDA cores (LACE_NO_TC=1: FP32 products
  folded into compensated sums), which sees identical Psi and W, so the
  difference is the tensor-core contraction's own error.

Measured values are printed (pytest -s).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_FP64, LACE_MIXED, LACE_SYM_AVG, Lace
from paper_1801_09263_gb300 import binding as B

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

S_THR = 1e-3


@pytest.fixture(scope="module")
def runs():
    sysm = synth.config2_water_like()
    n = sysm.n_occ
    with Lace(0, LACE_FP64) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, n, 0, True)
        piv = ctx.localize(2)
    out = {}
    mp = pytest.MonkeyPatch()
    try:
        for tc in (True, False):
            if tc:
                mp.delenv("LACE_NO_TC", raising=False)
            else:
                mp.setenv("LACE_NO_TC", "1")
            with Lace(0, LACE_MIXED) as ctx:
                ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
                ctx.load_orbitals(sysm.phi, n, 0, True)
                ctx.set_pivots(piv)
                npairs = ctx.screen(S_THR)
                S = ctx.get_matrix(B.MAT_OVERLAP_MODULI)
                pairs = ctx.get_pairs()
                ctx.apply_exchange(want_W=False)
                ctx.build_ace(LACE_SYM_AVG)
                M = ctx.get_matrix(B.MAT_EXCHANGE)
            out[tc] = dict(S=S, M=M, pairs=pairs, n=npairs)
    finally:
        mp.undo()
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi)
    _, _, w = O.scdm(g, occ, 2, pivots=piv)
    s_ref = O.overlap_moduli(g, w)
    return n, s_ref, out


def test_overlap_of_moduli_on_tensor_cores(runs):
    n, s_ref, out = runs
    S = out[True]["S"]
    off = ~np.eye(n, dtype=bool)
    d = np.diag(s_ref)
    bias = np.mean((np.diag(S) - d) / d)
    near = off & (s_ref >= 0.5 * S_THR) & (s_ref <= 2 * S_THR)
    rel_near = np.max(np.abs(S - s_ref)[near] / s_ref[near])
    print(f"S diagonal bias {bias:.3g}; max rel error in [S_thr/2, 2 S_thr] {rel_near:.3g} "
          f"({int(near.sum())} entries); max abs {np.max(np.abs(S - s_ref)):.3g}")
    assert abs(bias) < 2e-6
    assert rel_near < 1e-4
    assert np.max(np.abs(S - s_ref)) < 1e-5
    # kept pairs: identical to the oracle's screen outside a 1e-4 band around S_thr
    keep_ref = O.kept_pairs(s_ref, S_THR, n, 0)
    keep = np.zeros((n, n), dtype=bool)
    for i, j in out[True]["pairs"]:
        keep[i, j] = keep[j, i] = True
    band = np.abs(s_ref - S_THR) <= 1e-4 * S_THR
    assert not ((keep != keep_ref) & ~band).any()


def test_ace_matrix_on_tensor_cores_against_cuda_cores(runs):
    _, _, out = runs
    assert out[True]["n"] == out[False]["n"]
    Mt, Mc = out[True]["M"], out[False]["M"]
    bias = np.mean((np.diag(Mt) - np.diag(Mc)) / np.diag(Mc))
    rel = np.max(np.abs(Mt - Mc)) / np.max(np.abs(Mc))
    print(f"M' diagonal bias {bias:.3g}; max rel error {rel:.3g}")
    assert abs(bias) < 1e-6
    assert rel < 5e-6
