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
    # outputs start dirty (the call must clear them), allocated before the
    # calls so that nothing else allocates device memory between them
    outs = [(torch.full_like(d_psi, float("nan")),
             torch.full((n_occ, n_occ), float("nan"), dtype=torch.float64, device=dev)) for _ in range(2)]
    torch.cuda.synchronize(dev)
    for call, (d_W, d_e) in enumerate(outs):
        free_before = torch.cuda.mem_get_info(dev)[0]
        st = lib.lace_exchange_pairs_noalloc(cell.ctypes.data_as(C.c_void_p), *sysm.shape,
                                             C.c_void_p(d_psi.data_ptr()), n_occ, n_p,
                                             C.c_void_p(d_pairs.data_ptr()), len(pairs),
                                             C.c_void_p(d_W.data_ptr()), C.c_void_p(d_e.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
        assert st == 0, (call, lib.lace_status_string(st))
        torch.cuda.synchronize(dev)
        if call == 1:
            # after the first call (which may load the library's device code
            # and look up the array), a call takes no device memory at all
            assert torch.cuda.mem_get_info(dev)[0] == free_before
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
    dup = torch.tensor([[0, 1], [0, 1]], dtype=torch.int32, device=dev)  # the same pair twice
    assert lib.lace_exchange_pairs_noalloc(*args(dup, 2, (16, 16, 16))) == 1


def test_noalloc_rejects_a_pair_list_one_grid_short_of_fitting():
    """The 32 MiB array holds the flag, the FFT tables, the pair bitmap, the
    pair descriptors and at least one complex grid with its energy partials;
    a pair list 256 bytes of descriptors past that is refused (status 7)
    before anything is read or queued."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    lib = B.load_library()
    n, n_occ, n_p = 4, 1024, 8192
    r256 = lambda b: (b + 255) // 256 * 256
    seen = r256((n_occ * n_p + 31) // 32 * 4)
    fits = (32 << 20) - (256 + 16384 + seen + r256(n * 2 * 8) + n ** 3 * 16)  # descriptor bytes that still fit
    n_grids = (fits + 256) // 16
    n_pairs = 2 * n_grids
    # a real, in-range, duplicate-free list of that length (occupied x extra pairs)
    i = torch.arange(n_pairs, device=dev) % n_occ
    j = n_occ + torch.arange(n_pairs, device=dev) // n_occ
    assert int(j.max()) < n_p
    pairs = torch.stack([i, j], 1).to(torch.int32).contiguous()
    d_psi = torch.zeros((n_p, n, n, n), dtype=torch.float64, device=dev)
    d_W = torch.zeros_like(d_psi)
    d_e = torch.zeros((n_occ, n_occ), dtype=torch.float64, device=dev)
    cell = np.array([5.0, 5.0, 5.0])
    st = lib.lace_exchange_pairs_noalloc(cell.ctypes.data_as(C.c_void_p), n, n, n, C.c_void_p(d_psi.data_ptr()),
                                         n_occ, n_p, C.c_void_p(pairs.data_ptr()), n_pairs,
                                         C.c_void_p(d_W.data_ptr()), C.c_void_p(d_e.data_ptr()), None)
    assert st == 7, lib.lace_status_string(st)
