"""Launch plans of the out-of-place FFT passes, checked on the host.

The plans (radices, threads, register caps, shared memory) are compile-time
functions of the grid size in ``csrc/pairconv_spec2.cuh``; a host-only program
built from that header checks, for every size-specialised grid, that the plan
is a two-radix factorisation and that the planned CTAs fit one SM (threads,
per-sub-partition registers, shared memory).  No GPU is needed.
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
    assert len(lines) == 13 and all(line.endswith("ok") for line in lines), out.stdout
    # the 72^3 workload: radix 9 x 8, 576 threads, two CTAs per SM
    assert "n=72 plan=9x8 threads=576 ctas=2" in out.stdout
