"""Plane-wave front end on the device against the oracle's transforms.

The synthetic orbitals are band-limited to the cutoff sphere, so their
coefficients in the half-sphere basis represent them exactly: loading the
coefficients must give back the grid orbitals (then Loewdin as usual), and
the exchange W read back as coefficients must equal the oracle's W sampled
on the basis.  FP64 transforms in both precision modes; the mixed path
stores orbitals in FP32 (relative 1e-7).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_FP64, LACE_MIXED, Lace, LaceError
from paper_1801_09263_gb300 import binding as B

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def sysm():
    # non-cubic grid, odd axis, 6 occupied + 2 extras
    return synth.small_localized_system(31, (9.0, 10.0, 11.0), (24, 27, 30), 6.0, 4, 6, 2)


@pytest.mark.parametrize("prec", [LACE_FP64, LACE_MIXED], ids=["fp64", "mixed"])
def test_load_from_coefficients_and_read_back(sysm, prec):
    g = O.Grid(sysm.cell, sysm.shape)
    m = O.pw_basis(sysm.cell, sysm.ecut)
    coef = O.grid_to_pw(g, m, sysm.phi)
    assert relerr(O.pw_to_grid(g, m, coef), sysm.phi) < 1e-12  # band-limited: exact
    rep = 1e-12 if prec == LACE_FP64 else 2e-7
    with Lace(0, prec) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals_pw(coef, 6, 2, orthonormalize=False)
        assert relerr(ctx.get_orbitals(B.ORB_PSI), sysm.phi) < rep
        back = ctx.get_orbitals_pw(B.ORB_PSI, len(m))
        assert relerr(back, coef) < rep
        # orthonormalised, exchange, W as coefficients
        ctx.load_orbitals_pw(coef, 6, 2, orthonormalize=True)
        W, ex = ctx.apply_exchange()
        w_pw = ctx.get_orbitals_pw(B.ORB_W, len(m))
    occ = O.lowdin(g, sysm.phi[:6])
    extra = O.orthonormalize_extras(g, occ, sysm.phi[6:])
    W_ref, ex_ref, _ = O.apply_exchange(g, occ, extra, np.ones((6, 8), dtype=bool))
    tol = 1e-10 if prec == LACE_FP64 else 2e-5
    assert relerr(W, W_ref) < tol
    assert relerr(w_pw, O.grid_to_pw(g, m, W_ref)) < tol
    assert abs(ex - ex_ref) <= (1e-6 if prec == LACE_FP64 else 1e-5)


def test_sphere_larger_than_the_grid_is_rejected(sysm):
    m = O.pw_basis(sysm.cell, 40.0)
    with Lace(0, LACE_FP64) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, 40.0)
        with pytest.raises(LaceError):
            ctx.load_orbitals_pw(np.zeros((2, len(m)), dtype=complex), 2, 0)
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        with pytest.raises(LaceError):  # wrong coefficient count
            ctx.load_orbitals_pw(np.zeros((2, len(m)), dtype=complex), 2, 0)
