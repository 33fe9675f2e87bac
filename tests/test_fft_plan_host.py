"""Launch plans of the out-of-place FFT passes, checked on the host.

The plans (radices, threads, register caps, shared memory) are compile-time
functions of the grid size in ``csrc/pairconv_spec2.cuh`` (one complex grid
per CTA) and ``csrc/pairconv_pair.cuh`` (two grids per CTA in packed FP32
pairs, where both paired planes fit in shared memory); a host-only program
built from those headers checks, for every size-specialised grid, that the
plan is a two-radix factorisation and that the planned CTAs fit one SM
(threads, per-sub-partition registers, shared memory).  No GPU is needed.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1801_09263_gb300", "csrc")


def test_out_of_place_pass_plans_fit_one_sm(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "fft_plan_check"
    src = os.path.join(ROOT, "tests", "fft_plan_check.cu")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                        "-I", CSRC, "-I",
                        os.path.join(ROOT, "include"), src, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    lines = out.stdout.strip().splitlines()
    assert len(lines) == 11 + 9 and all(line.endswith("ok") for line in lines), out.stdout
    # the 72^3 workload: radix 9 x 8; one grid per CTA: 576 threads, two CTAs
    # per SM; two grids per CTA: 672 threads (one round of the 648 radix-8
    # butterflies), one CTA per SM (188 KB of paired planes and K slab), 80 registers
    assert "n=72 plan=9x8 threads=576 ctas=2" in out.stdout
    assert "pair n=72 plan=9x8 threads=672 ctas=1 regs=80" in out.stdout
    assert not any(line.startswith("pair n=96") for line in lines)  # two paired 96^2 planes do not fit
