"""Error paths of the C ABI that need a GPU: a Cholesky failure of M' and a
bounded device wait that runs out.  Neither faults, traps or hangs the GPU:
the failing input is made on the host, and the wait gives up through its own
time limit and reports through a flag the host reads.
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_FP64, LACE_MIXED, Lace, LaceError
from paper_1801_09263_gb300 import binding as B

pytestmark = pytest.mark.gpu

NOT_PD, TIMEOUT = 5, 6


@pytest.mark.parametrize("prec", [LACE_FP64, LACE_MIXED], ids=["fp64", "mixed"])
def test_cholesky_failure_keeps_the_previous_ace_projector(prec):
    """Sec. 2 factors -M' = L L^T and argues M' stays definite for small
    truncations; a threshold above 1 drops every pair (S_ik <= 1), so W = 0,
    M' = 0 and the factorisation meets a zero pivot.  The call must return
    LACE_ERR_NOT_PD and leave the projector built before it untouched."""
    sysm = synth.small_localized_system(31, (11.0, 11.0, 11.0), (24, 24, 24), 10.0, 6, 8)
    g = O.Grid(sysm.cell, sysm.shape)
    probe = np.random.default_rng(5).standard_normal((2,) + sysm.shape)
    with Lace(0, prec) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, 8, 0, True)
        ctx.localize(2)
        ctx.screen(1e-3)
        W, _ = ctx.apply_exchange()
        ctx.build_ace()
        k0 = ctx.apply_ace(probe)
        L0 = ctx.get_matrix(B.MAT_CHOLESKY)
        xi0 = ctx.get_orbitals(B.ORB_XI)
        assert ctx.screen(2.0) == 0
        W2, ex2 = ctx.apply_exchange()
        assert ex2 == 0.0 and not W2.any()
        with pytest.raises(LaceError) as e:
            ctx.build_ace()
        assert e.value.status == NOT_PD
        # the oracle's factorisation fails on the same M' (zero matrix)
        m = O.symmetrize(g.dv * (ctx.get_orbitals(B.ORB_PSI).reshape(8, -1) @ W2.reshape(8, -1).T))
        assert not m.any()
        with pytest.raises(np.linalg.LinAlgError):
            np.linalg.cholesky(-m)
        # projector, factor and application unchanged, bit for bit
        assert np.array_equal(ctx.get_matrix(B.MAT_CHOLESKY), L0)
        assert np.array_equal(ctx.get_orbitals(B.ORB_XI), xi0)
        assert np.array_equal(ctx.apply_ace(probe), k0)
        # and a later successful build replaces it (the same operator again,
        # up to the order of the W accumulations)
        ctx.screen(1e-3)
        ctx.apply_exchange()
        ctx.build_ace()
        k3 = ctx.apply_ace(probe)
        assert np.max(np.abs(k3 - k0)) <= (1e-12 if prec == LACE_FP64 else 1e-5) * np.max(np.abs(k0))


@pytest.mark.parametrize("prec", [LACE_FP64, LACE_MIXED], ids=["fp64", "mixed"])
def test_grid_barrier_wait_that_runs_out_returns_timeout(prec):
    """The pivoted QR of SCDM (Sec. 2) runs as one persistent launch whose
    CTAs meet at a time-limited grid barrier every pivot step.  With the
    limit set to 0 every wait that has to wait gives up at once: the CTAs
    leave the kernel, lace_localize returns LACE_ERR_TIMEOUT, and after the
    default limit is restored the same context localises to the same pivots
    as a fresh one."""
    # 48^3 grid: 24^3 = 13,824 subsample columns spread over ~100 CTAs
    sysm = synth.small_localized_system(41, (14.0, 14.0, 14.0), (48, 48, 48), 12.0, 24, 32)
    with Lace(0, prec) as ref:
        ref.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ref.load_orbitals(sysm.phi, 32, 0, True)
        piv_ref = ref.localize(2)
    with Lace(0, prec) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, 32, 0, True)
        ctx.set_wait_limit(0.0)
        with pytest.raises(LaceError) as e:
            ctx.localize(2)
        assert e.value.status == TIMEOUT
        with pytest.raises(LaceError) as e:  # not localised: no SCDM rotation to read
            ctx.get_matrix(B.MAT_SCDM_U)
        assert e.value.status == 2
        ctx.set_wait_limit(2.0)
        piv = ctx.localize(2)
        assert np.array_equal(piv, piv_ref)
        with pytest.raises(LaceError) as e:
            ctx.set_wait_limit(-1.0)
        assert e.value.status == 1
