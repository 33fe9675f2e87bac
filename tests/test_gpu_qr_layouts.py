"""SCDM pivoted QR (Sec. 2) on every row layout of the persistent FP32 kernel.

The mixed-precision QR keeps the subsample matrix on chip: 1 to 16 lanes per
column hold 32 or 64 rows each in registers (512 threads a CTA), and the
columns a CTA cannot hold in registers sit in shared memory.  Each case below
picks a grid and orbital count that lands on one layout (with and without
shared-memory columns) and checks the pivots against the FP64 oracle:
replaying the oracle's exact Gram-Schmidt steps with the GPU's pivot order,
every choice must be within 1e-4 of the largest residual norm (the FP32
kernel's rounding; a valid Businger-Golub order has every ratio 1), and a
second run must pick the same pivots.
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_MIXED, Lace

pytestmark = pytest.mark.gpu

CASES = [  # (grid n, cell L, ecut, centres, orbitals): rows per lane x lanes per column, columns in shared memory
    (48, 16.0, 20.0, 20, 24),     # 32 x 1, registers only
    (96, 28.0, 30.0, 20, 24),     # 32 x 1, 110,592 columns: shared memory too
    (64, 20.0, 30.0, 48, 60),     # 64 x 1, registers only
    (72, 23.5, 30.0, 80, 100),    # 64 x 2, shared memory too
    (48, 16.0, 20.0, 100, 140),   # 64 x 4, registers only
    (64, 20.0, 30.0, 120, 160),   # 64 x 4, shared memory too
    (48, 16.0, 20.0, 200, 300),   # 64 x 8, shared memory too
]


@pytest.mark.parametrize("n,L,ecut,nc,no", CASES, ids=[f"{c[0]}^3x{c[4]}" for c in CASES])
def test_pivots_are_a_valid_qrcp_order(n, L, ecut, nc, no):
    sysm = synth.small_localized_system(900 + no, (L, L, L), (n, n, n), ecut, nc, no)
    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi)
    with Lace(0, LACE_MIXED) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, no, 0, True)
        piv = ctx.localize(2)
        piv2 = ctx.localize(2)
    assert np.array_equal(piv, piv2)
    assert len(set(int(p) for p in piv)) == no
    sub = O.subsample_indices(g.shape, 2)
    pos = {int(v): k for k, v in enumerate(sub)}
    cols = [pos[int(p)] for p in piv]
    ratios = O.qrcp_pivot_ratios(occ.reshape(no, -1)[:, sub], cols)
    assert ratios.min() >= 1 - 1e-4, (ratios.min(), int(np.argmin(ratios)))
