"""Batched uneven instances on the device.

Eight systems with different cells, grids (one odd size on the generic FFT
radices, the others with specialised passes, among them 50^3 and 54^3 whose
rows are not 16-byte multiples) and orbital counts run through one
lace_batch: the first run is eager, the second
captures the CUDA graph, later runs replay it.  Each instance's E_x, W and
xi must match a single-system context on the same orbitals (the same method
on the single-system kernels) within the mixed-precision tolerances
(|dE_x| <= 1e-5 Ha, 2e-5 relative on W and xi); graph replays must agree
with the eager run; a tiny scratch pool (several chunks, several launches)
must give the same results; one instance at S_thr = 0 is checked against
the FP64 oracle (E_x is then independent of the SCDM rotation).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_1801_09263_gb300 import LACE_MIXED, Batch, Lace
from paper_1801_09263_gb300 import binding as B

pytestmark = pytest.mark.gpu

INST = [  # L, n, ecut, n_occ, s_thr
    (10.0, 24, 12.0, 8, 0.0),
    (12.0, 32, 14.0, 20, 1e-3),
    (11.0, 45, 30.0, 12, 1e-3),
    (14.0, 48, 20.0, 24, 1e-3),
    (13.0, 36, 16.0, 16, 1e-3),
    (15.0, 32, 10.0, 30, 1e-3),
    (14.0, 50, 22.0, 18, 1e-3),
    (15.0, 54, 22.0, 14, 1e-3),
]


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def systems():
    out = []
    for k, (L, n, ecut, no, thr) in enumerate(INST):
        s = synth.ServingSystem(k, (L, L, L), (n, n, n), ecut, no, 500 + k)
        out.append((s, thr, synth.serving_orbitals(s)))
    return out


def single(s, thr, phi):
    with Lace(0, LACE_MIXED) as c:
        c.set_cell(s.cell, s.shape, s.ecut)
        c.load_orbitals(phi, s.n_occ, 0, True)
        c.localize(2)
        c.screen(thr)
        W, ex = c.apply_exchange()
        c.build_ace()
        return dict(ex=ex, W=W, xi=c.get_orbitals(B.ORB_XI), pairs=c.get_pairs())


@pytest.fixture(scope="module")
def batch_runs():
    sy = systems()
    phis = [p.copy() for _, _, p in sy]
    out = {}
    with Batch([(s.cell, s.shape, s.ecut, s.n_occ, thr) for s, thr, _ in sy]) as b:
        for q, p in enumerate(phis):
            b.set_orbitals(q, p)
        res = []
        for _ in range(3):  # eager, capture, replay
            ex, st = b.run()
            res.append((ex.copy(), st.copy()))
        out["runs"] = res
        out["info"] = b.info()
        views = [b.context(q) for q in range(len(sy))]
        out["W"] = [v.get_orbitals(B.ORB_W) for v in views]
        out["xi"] = [v.get_orbitals(B.ORB_XI) for v in views]
        out["pairs"] = [v.get_pairs() for v in views]
        out["piv"] = [v.get_pivots() for v in views]
        # drift the orbitals (out of their span) and replay the graph
        for p in phis:
            synth.perturb_in_place(p, 3e-2)
        ex2, st2 = b.run()
        out["perturbed"] = (ex2, st2, [p.copy() for p in phis])
        out["info2"] = b.info()
    return sy, out


def test_batch_matches_single_system_contexts(batch_runs):
    sy, out = batch_runs
    ex, st = out["runs"][0]
    assert (st == 0).all(), st
    for q, (s, thr, phi) in enumerate(sy):
        r = single(s, thr, phi)
        assert len(out["pairs"][q]) == len(r["pairs"])
        assert abs(ex[q] - r["ex"]) <= 1e-5, (q, ex[q], r["ex"])
        assert relerr(out["W"][q], r["W"]) <= 2e-5
        assert relerr(out["xi"][q], r["xi"]) <= 2e-5


def test_graph_replays_agree_with_the_eager_run(batch_runs):
    _, out = batch_runs
    ex0 = out["runs"][0][0]
    for ex, st in out["runs"][1:]:
        assert (st == 0).all()
        assert np.max(np.abs(ex - ex0)) <= 1e-6
    info = out["info"]
    assert info["graph_replays"] >= 2 and info["threads"] in (128, 256, 512) and info["chunks"] >= 1
    assert info["launches"] > 0 and info["pairconv_ms"] > 0


def test_graph_replay_with_new_orbitals(batch_runs):
    sy, out = batch_runs
    ex2, st2, phis = out["perturbed"]
    assert (st2 == 0).all()
    assert out["info2"]["graph_replays"] >= 3
    for q in (0, 2, 5):
        s, thr, _ = sy[q]
        r = single(s, thr, phis[q])
        assert abs(ex2[q] - r["ex"]) <= 1e-5
    assert np.max(np.abs(ex2 - out["runs"][0][0])) > 1e-5  # the drift changed E_x


def test_unscreened_instance_matches_the_fp64_oracle(batch_runs):
    sy, out = batch_runs
    s, thr, phi = sy[0]
    assert thr == 0.0
    g = O.Grid(s.cell, s.shape)
    occ = O.lowdin(g, phi)
    _, ex_ref, _ = O.apply_exchange(g, occ, None, np.ones((s.n_occ, s.n_occ), dtype=bool))
    assert abs(out["runs"][0][0][0] - ex_ref) <= 1e-5


@pytest.mark.parametrize("q", [3, 4])
def test_screened_instance_matches_the_fp64_oracle(batch_runs, q):
    """A localised, screened instance (S_thr = 1e-3) against the oracle on the
    instance's own SCDM points: the points must be a valid pivoted-QR order
    of the oracle's canonical orbitals (every choice within 1e-4 of the
    largest residual norm, the FP32 QR's rounding), the kept pair set must
    equal the oracle's outside a 1e-5 band around the threshold, and E_x, W
    and xi must match the oracle's localised exchange and ACE build
    (Sec. 2, Eqs. 2-5 and the Cholesky form of ACE)."""
    sy, out = batch_runs
    s, thr, phi = sy[q]
    assert thr > 0
    n = s.n_occ
    g = O.Grid(s.cell, s.shape)
    occ = O.lowdin(g, phi)
    piv = out["piv"][q]
    sub = O.subsample_indices(s.shape, 2)
    col = {int(p): k for k, p in enumerate(sub)}
    ratios = O.qrcp_pivot_ratios(occ.reshape(n, -1)[:, sub], [col[int(p)] for p in piv])
    assert ratios.min() >= 1.0 - 1e-4, ratios.min()
    _, _, w = O.scdm(g, occ, 2, pivots=piv)
    S = O.overlap_moduli(g, w)
    keep = np.zeros((n, n), dtype=bool)
    for i, j in out["pairs"][q]:
        keep[i, j] = keep[j, i] = True
    outside = np.abs(S - thr) > 1e-5 * thr
    assert np.array_equal(keep[outside], (S >= thr)[outside])
    assert keep.sum() < n * n  # the screen dropped pairs
    W_ref, ex_ref, _ = O.apply_exchange(g, w, None, keep)
    xi_ref, _, _ = O.ace_build(g, w, W_ref)
    assert abs(out["runs"][0][0][q] - ex_ref) <= 1e-5
    assert relerr(out["W"][q], W_ref) <= 2e-5
    assert relerr(out["xi"][q], xi_ref) <= 5e-5


def test_small_scratch_pool_gives_the_same_results(batch_runs, monkeypatch):
    sy, out = batch_runs
    monkeypatch.setenv("LACE_BATCH_POOL_MB", "2")
    with Batch([(s.cell, s.shape, s.ecut, s.n_occ, thr) for s, thr, _ in sy]) as b:
        for q, (_, _, p) in enumerate(sy):
            b.set_orbitals(q, p)
        for _ in range(2):
            ex, st = b.run()
            assert (st == 0).all()
            assert np.max(np.abs(ex - out["runs"][0][0])) <= 1e-6
        assert b.info()["chunks"] > 1


def test_per_instance_mode_matches_the_persistent_kernel(batch_runs, monkeypatch):
    """The per-instance mode (single-system passes, re-captured every run)
    against the persistent multi-instance kernel and single contexts."""
    sy, out = batch_runs
    monkeypatch.setenv("LACE_BATCH_MODE", "per_instance")
    phis = [p.copy() for _, _, p in sy]
    with Batch([(s.cell, s.shape, s.ecut, s.n_occ, thr) for s, thr, _ in sy]) as b:
        for q, p in enumerate(phis):
            b.set_orbitals(q, p)
        for _ in range(3):  # eager, capture, re-capture
            ex, st = b.run()
            assert (st == 0).all()
            assert np.max(np.abs(ex - out["runs"][0][0])) <= 1e-5
        info = b.info()
        assert info["mode"] == "per_instance" and info["graph_replays"] >= 2
        assert info["tune_ms"]["per_instance"] > 0
        for p in phis:
            synth.perturb_in_place(p, 3e-2)
        ex2, st2 = b.run()
        assert (st2 == 0).all()
        for q in (0, 2, 5):
            s, thr, _ = sy[q]
            assert len(b.context(q).get_pairs()) == len(single(s, thr, phis[q])["pairs"])
            assert abs(ex2[q] - single(s, thr, phis[q])["ex"]) <= 1e-5


@pytest.mark.parametrize("shape", ["256x2", "512x1", "512x2"])
def test_every_persistent_launch_shape_matches(batch_runs, monkeypatch, shape):
    """The persistent kernel in each of its shapes with size-specialised
    bodies (thread groups of 128-512 threads sharing a CTA, each on its own
    plane or slab): E_x, W and xi against the first run of the batch (which
    the autotuner may have given to either mode)."""
    sy, out = batch_runs
    monkeypatch.setenv("LACE_BATCH_SHAPE", shape)
    with Batch([(s.cell, s.shape, s.ecut, s.n_occ, thr) for s, thr, _ in sy]) as b:
        for q, (_, _, p) in enumerate(sy):
            b.set_orbitals(q, p)
        for _ in range(2):  # eager, capture
            ex, st = b.run()
            assert (st == 0).all(), st
            assert np.max(np.abs(ex - out["runs"][0][0])) <= 1e-5
        info = b.info()
        assert info["mode"] == "persistent"
        assert f'{info["threads"]}x{info["ctas_per_sm"]}' == shape
        for q in range(len(sy)):
            v = b.context(q)
            assert relerr(v.get_orbitals(B.ORB_W), out["W"][q]) <= 2e-5
            assert relerr(v.get_orbitals(B.ORB_XI), out["xi"][q]) <= 2e-5
