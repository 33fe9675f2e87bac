"""The allocation-free exchange call matches lace_apply_exchange.

lace_exchange_pairs_noalloc serves callers that cannot allocate device
memory at the point of use (latency-critical loops where cudaMalloc would
synchronise the device, or programs whose device memory belongs to their own
pool allocator).  It takes its scratch from a fixed array inside the library,
so two calls in a row must both reproduce the context-based result: the
second call must not see anything the first one left behind.  This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_1801_09263_gb300 import LACE_FP64, Lace
from paper_1801_09263_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_noalloc_exchange_matches_context_call_twice():
    torch = pytest.importorskip("torch")
    sysm = synth.small_localized_system(77, (13.0, 13.0, 13.0), (36, 36, 36), 12.0, 14, 20, 4)
    n_occ, n_p = sysm.n_occ, sysm.n_occ + sysm.n_extra
    with Lace(0, LACE_FP64) as ctx:
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        ctx.load_orbitals(sysm.phi, n_occ, sysm.n_extra, True)
        ctx.localize(2)
        ctx.screen(1e-3)
        W_ref, ex_ref = ctx.apply_exchange()
        e_ref = ctx.get_matrix(B.MAT_PAIR_ENERGY)
        psi = ctx.get_orbitals(B.ORB_PSI)
        pairs = ctx.get_pairs()
    assert 0 < len(pairs) < n_occ * (n_occ + 1) // 2 + n_occ * sysm.n_extra  # screening dropped some pairs

    dev = torch.device("cuda", 0)
    d_psi = torch.from_numpy(psi).to(dev)
    d_pairs = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).to(dev)
    cell = np.ascontiguousarray(sysm.cell, dtype=np.float64)
    lib = B.load_library()
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        d_W = torch.full_like(d_psi, float("nan"))  # outputs start dirty: the call must clear them
        d_e = torch.full((n_occ, n_occ), float("nan"), dtype=torch.float64, device=dev)
        st = lib.lace_exchange_pairs_noalloc(cell.ctypes.data_as(C.c_void_p), *sysm.shape,
                                             C.c_void_p(d_psi.data_ptr()), n_occ, n_p,
                                             C.c_void_p(d_pairs.data_ptr()), len(pairs),
                                             C.c_void_p(d_W.data_ptr()), C.c_void_p(d_e.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
        assert st == 0, (call, lib.lace_status_string(st))
        torch.cuda.synchronize(dev)
        W = d_W.cpu().numpy()
        e = d_e.cpu().numpy()
        assert np.abs(W - W_ref).max() <= 1e-10 * np.abs(W_ref).max(), call
        assert np.abs(e - e_ref).max() <= 1e-10 * np.abs(e_ref).max(), call
        assert abs(-0.5 * e.sum() - ex_ref) <= 1e-6, call


def test_noalloc_rejects_bad_pairs_and_sizes():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    lib = B.load_library()
    cell = np.array([10.0, 10.0, 10.0])
    d_psi = torch.zeros((2, 16, 16, 16), dtype=torch.float64, device=dev)
    d_W = torch.zeros_like(d_psi)
    d_e = torch.zeros((2, 2), dtype=torch.float64, device=dev)
    bad = torch.tensor([[0, 1], [1, 0]], dtype=torch.int32, device=dev)  # (1, 0): i > j for occupied j
    args = lambda pairs, n, shape: (cell.ctypes.data_as(C.c_void_p), *shape, C.c_void_p(d_psi.data_ptr()), 2, 2,
                                    C.c_void_p(pairs.data_ptr()), n, C.c_void_p(d_W.data_ptr()),
                                    C.c_void_p(d_e.data_ptr()), None)
    assert lib.lace_exchange_pairs_noalloc(*args(bad, 2, (16, 16, 16))) == 1
    assert lib.lace_exchange_pairs_noalloc(*args(bad, 1, (16, 16, 7))) == 7  # 7 is not 2^a 3^b 5^c
    assert lib.lace_exchange_pairs_noalloc(*args(bad, 1, (128, 128, 128))) == 7  # FP64 planes exceed shared memory
    assert lib.lace_exchange_pairs_noalloc(*args(bad, 1, (16, 16, 16))) == 0
