"""The C-ABI library builds for sm_103a, loads, and exports every declared call (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

import paper_1801_09263_gb300 as lace
from paper_1801_09263_gb300.build import build


@pytest.fixture(scope="module")
def libpath():
    return build()


def test_library_builds_and_exports_declared_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    declared = lace.exported_symbols()
    assert len(declared) >= 20
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared in include/lace.h but not exported: {missing}"


def test_library_loads_and_status_strings(libpath):
    lib = lace.load_library()
    assert lib.lace_status_string(0) == b"ok"
    assert lib.lace_status_string(5) == b"matrix not positive definite"
    assert lib.lace_status_string(2) == b"call made out of order"


def test_destroy_null_is_ok(libpath):
    lib = lace.load_library()
    assert lib.lace_destroy(None) == 0


def test_create_rejects_bad_precision(libpath):
    lib = lace.load_library()
    h = ctypes.c_void_p()
    assert lib.lace_create(ctypes.byref(h), 0, 7) == 1  # LACE_ERR_ARG, checked before any CUDA call


def test_axis_plans_cover_supported_sizes():
    # every 2^a 3^b 5^c size in [4, 128] has a plan of at most 4 register radices
    from paper_1801_09263_gb300.build import CSRC
    src = open(os.path.join(CSRC, "pairconv.cu")).read()
    radices = [16, 12, 10, 9, 8, 6, 5, 4, 3, 2]
    assert "static const int kRadices[] = {16, 12, 10, 9, 8, 6, 5, 4, 3, 2};" in src

    def plan(n, depth=4):
        if n == 1:
            return []
        if depth == 0:
            return None
        for r in radices:
            if n % r == 0:
                sub = plan(n // r, depth - 1)
                if sub is not None:
                    return [r] + sub
        return None

    for n in range(4, 129):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            assert plan(n) is not None, n
