"""Index algebra of the out-of-place FFT passes, restated in numpy.

The CUDA passes (``csrc/pairconv_spec2.cuh``) run each axis as two register
radix stages of a Stockham FFT, and pass B runs the x axis as decimation in
time forward and decimation in frequency inverse so that the second forward
stage, the product with K and the first inverse stage share registers:
for n = A B, x index n1 + A n2 and k index k2 + B k1,

    X[k2 + B k1] = sum_n1 w_A^{n1 k1} w_n^{n1 k2} sum_n2 w_B^{n2 k2} x[n1 + A n2]
    x[n1 + A n2] = sum_k2 w_B^{-n2 k2} w_n^{-n1 k2} sum_k1 w_A^{-n1 k1} Y[k2 + B k1].

These tests replay the same element maps (butterfly i reads i + t n/R and
writes (i - k) R + k + s P; the middle writes n1 B + k2, the last stage reads
it back) on random data and compare with numpy's FFT, for every radix plan of
the size-specialised grids.
"""
import numpy as np
import pytest

RADICES = (2, 3, 4, 5, 6, 8, 9, 10, 12, 16)
SIZES = (24, 32, 36, 40, 48, 50, 54, 60, 64, 72, 80, 96, 100)


def plan2(n):
    """Two register radices r1 r2 = n with the largest smaller factor (r1 first found)."""
    best, best_min = None, 0
    for r1 in range(16, 1, -1):
        if r1 not in RADICES or n % r1:
            continue
        r2 = n // r1
        if r2 in RADICES and min(r1, r2) > best_min:
            best, best_min = (r1, r2), min(r1, r2)
    return best


def dft(v, sign):
    r = len(v)
    t = np.arange(r)
    return np.exp(sign * 2j * np.pi * np.outer(t, t) / r) @ v


def stockham_stage(x, radix, p, sign):
    """One out-of-place radix stage: butterfly i reads i + t n/R, twiddle w^{t k}, writes (i-k) R + k + s p."""
    n = len(x)
    tn = n // radix
    w = np.exp(-2j * np.pi * np.arange(n) / n)
    y = np.empty(n, complex)
    for i in range(tn):
        v = np.array([x[i + t * tn] for t in range(radix)])
        k = i % p if p > 1 else 0
        if p > 1:
            tw = np.array([w[(t * k * (n // (p * radix))) % n] for t in range(radix)])
            v = v * (np.conj(tw) if sign > 0 else tw)
        v = dft(v, sign)
        base = (i - k) * radix + k
        for s in range(radix):
            y[base + s * p] = v[s]
    return y


@pytest.mark.parametrize("n", SIZES)
def test_two_stage_stockham_is_the_dft(n):
    r1, r2 = plan2(n)
    x = np.random.default_rng(n).standard_normal(n) + 1j * np.random.default_rng(n + 1).standard_normal(n)
    fwd = stockham_stage(stockham_stage(x, r1, 1, -1), r2, r1, -1)
    assert np.allclose(fwd, np.fft.fft(x), atol=1e-9 * n)
    inv = stockham_stage(stockham_stage(x, r1, 1, +1), r2, r1, +1)
    assert np.allclose(inv, np.fft.ifft(x) * n, atol=1e-9 * n)


@pytest.mark.parametrize("n", SIZES)
def test_pass_b_middle_is_the_convolution(n):
    r1, r2 = plan2(n)
    rb, ra = r2, r1  # the middle (forward stage 2, K, inverse stage 1) takes radix ra
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    kk = rng.standard_normal(n)
    w = np.exp(-2j * np.pi * np.arange(n) / n)
    b0 = stockham_stage(x, rb, 1, -1)  # y[n1 rb + k2]
    b1 = np.empty(n, complex)
    for k2 in range(rb):
        v = np.array([b0[k2 + t * rb] * (w[t * k2] if t else 1.0) for t in range(ra)])
        v = dft(v, -1) * np.array([kk[k2 + s * rb] for s in range(ra)])
        v = dft(v, +1)
        for n1 in range(ra):
            b1[n1 * rb + k2] = v[n1] * (np.conj(w[n1 * k2]) if n1 else 1.0)
    out = np.empty(n, complex)
    for n1 in range(ra):
        v = dft(np.array([b1[n1 * rb + t] for t in range(rb)]), +1)
        for s in range(rb):
            out[n1 + ra * s] = v[s]
    assert np.allclose(out, np.fft.ifft(kk * np.fft.fft(x)) * n, atol=1e-9 * n)
