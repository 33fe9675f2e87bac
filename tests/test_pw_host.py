"""Plane-wave basis and grid-from-cutoff of the library (host-side calls; no GPU).

The library's basis must be the oracle's, element by element and in order,
and lace_grid_for_cutoff must return the smallest 2/3/5-smooth sizes that hold
the cutoff sphere without folding.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_09263_gb300 import binding as B


@pytest.mark.parametrize("cell,ecut", [((10.0, 10.0, 10.0), 20.0), ((7.0, 8.0, 9.5), 6.0),
                                       ((23.5, 23.5, 23.5), 10.0), ((5.0, 11.0, 6.5), 13.0)])
def test_basis_equals_oracle(cell, ecut):
    assert np.array_equal(B.pw_basis(cell, ecut), O.pw_basis(cell, ecut))


def _smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


@pytest.mark.parametrize("cell,ecut", [((10.0, 10.0, 10.0), 20.0), ((23.5, 23.5, 23.5), 40.0),
                                       ((7.0, 8.0, 9.5), 6.0)])
def test_grid_for_cutoff_is_the_smallest_that_holds_the_sphere(cell, ecut):
    dims = B.grid_for_cutoff(cell, ecut)
    m = O.pw_basis(cell, ecut)
    for a in range(3):
        mmax = int(np.max(np.abs(m[:, a])))
        assert 2 * mmax < dims[a] and _smooth(dims[a])
        assert all(not _smooth(k) for k in range(2 * mmax + 1, dims[a]))
