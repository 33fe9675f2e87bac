"""Write ace96_oracle_sample.json: FP64 oracle values of the ACE workload.

Workload: the water-like system of synth.config3_water_like_with_extras
(L = 23.5 bohr, 96^3 grid, 256 occupied + 128 extra orbitals, E_cut = 40 Ha),
SCDM on the stride-2 subsample, S_thr = 1e-3, average symmetrisation.

Every value is computed by oracle/ alone (Loewdin, extras orthonormalised
against the occupied set, pivoted QR, SCDM rotation, overlap of moduli,
kept pairs, exchange of all 384 targets, ACE build and ACE apply; Sec. 2,
Eqs. 2-7).  Stored: the oracle's pivots (so the library can be run on the
same localised set), the kept-pair count, E_x, and K_ACE psi of the eight
seeded probes (numpy default_rng(11), standard normal, shape (8, 96, 96, 96))
on 512 seeded sample points each, with each probe's largest |K_ACE psi| over
the whole grid (the scale of the relative error).

Run from the repository root:  python tests/golden/make_ace96_oracle.py
It takes several minutes of host time (about 35,000 FP64 pair potentials).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ace96_oracle_sample.json")
S_THR = 1e-3
N_PROBES, PROBE_SEED = 8, 11
N_SAMPLE, SAMPLE_SEED = 512, 12


def main() -> None:
    t0 = time.time()
    sysm = synth.config3_water_like_with_extras()
    g = O.Grid(sysm.cell, sysm.shape)
    n_occ, n_extra = sysm.n_occ, sysm.n_extra
    occ = O.lowdin(g, sysm.phi[:n_occ])
    extra = O.orthonormalize_extras(g, occ, sysm.phi[n_occ:])
    piv, _, w = O.scdm(g, occ, 2)
    print(f"scdm {time.time() - t0:.0f} s", flush=True)
    s = O.overlap_moduli(g, w)
    keep = O.kept_pairs(s, S_THR, n_occ, n_extra)
    iu = np.triu_indices(n_occ)
    n_pairs = int(keep[:, :n_occ][iu].sum() + keep[:, n_occ:].sum())
    # S values closest to the threshold (a reader can see how near a tie is)
    off = s[:n_occ, :n_occ][np.triu_indices(n_occ, 1)]
    gap = float(np.min(np.abs(off - S_THR)) / S_THR)
    psi = np.concatenate([w, extra])
    W, ex, _ = O.apply_exchange(g, w, extra, keep)
    print(f"exchange {time.time() - t0:.0f} s, E_x = {ex:.12f}", flush=True)
    xi, _, _ = O.ace_build(g, psi, W)
    probe = np.random.default_rng(PROBE_SEED).standard_normal((N_PROBES,) + tuple(sysm.shape))
    k = O.ace_apply(g, xi, probe).reshape(N_PROBES, -1)
    pts = np.random.default_rng(SAMPLE_SEED).choice(g.ng, size=N_SAMPLE, replace=False)
    pts.sort()
    data = {
        "what": "FP64 oracle values of the 96^3 ACE workload (synth.config3_water_like_with_extras), "
                "written by tests/golden/make_ace96_oracle.py from oracle/ only",
        "paper": "arXiv:1801.09263 Sec. 2: SCDM localisation, Eq. 4 screening, Eq. 2 exchange with the "
                 "truncation of Eq. 5, ACE matrix Eq. 3 / Eq. 7 (average symmetrisation) and its Cholesky form",
        "s_thr": S_THR,
        "stride": 2,
        "pivots": [int(p) for p in piv],
        "n_pairs": n_pairs,
        "min_rel_gap_of_S_to_threshold": gap,
        "E_x_Ha": float(ex),
        "probe": {"seed": PROBE_SEED, "count": N_PROBES, "dist": "standard normal, shape (8, 96, 96, 96)"},
        "sample_points": [int(p) for p in pts],
        "sample_seed": SAMPLE_SEED,
        "k_ace_max_abs": [float(np.abs(k[q]).max()) for q in range(N_PROBES)],
        "k_ace_sample": [[float(v) for v in k[q, pts]] for q in range(N_PROBES)],
    }
    with open(OUT, "w") as f:
        json.dump(data, f, indent=0)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
