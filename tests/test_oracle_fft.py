"""Pins for the oracle's own FFT (Sec. III-B transforms), no GPU needed.

The brute-force DFT is pinned to closed forms (delta -> ones, pure tone ->
scaled delta); the Stockham FFT is pinned to the brute-force DFT, Parseval,
Hermitian symmetry, invertibility and, as a library special case, numpy.fft.
"""

import numpy as np
import pytest

from oracle import fft as F

SIZES = [1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 48, 96]


def test_brute_dft_closed_forms():
    for n in (1, 2, 3, 6, 8, 12):
        d = np.zeros(n, complex)
        d[0] = 1.0
        assert np.allclose(F.dft_brute(d), np.ones(n), atol=1e-14)
        for m in range(n):
            x = np.exp(2j * np.pi * m * np.arange(n) / n)
            X = F.dft_brute(x)
            ref = np.zeros(n, complex)
            ref[m] = n
            assert np.allclose(X, ref, atol=1e-12)
            # inverse of a scaled delta is the tone
            assert np.allclose(F.dft_brute(ref, inverse=True), x, atol=1e-13)


@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_brute(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
    scale = np.sqrt(n)
    assert np.max(np.abs(F.fft(x) - F.dft_brute(x))) < 1e-13 * scale * 10
    assert np.max(np.abs(F.fft(x, inverse=True) - F.dft_brute(x, inverse=True))) < 1e-14 * 10


def test_fft3_mixed_sizes_vs_brute():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 4, 12))            # [z, y, x]
    ref = x.astype(complex)
    for ax in (2, 1, 0):
        ref = F.dft_brute(ref, axis=ax)
    assert np.max(np.abs(F.fft3(x) - ref)) < 1e-12


@pytest.mark.parametrize("n", [16, 48, 96])
def test_parseval_and_hermitian(n):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, n))
    X = F.fft(x)
    assert np.allclose(np.sum(x * x, axis=1), np.sum(np.abs(X) ** 2, axis=1) / n, rtol=1e-13)
    k = np.arange(n)
    assert np.max(np.abs(X[:, (-k) % n] - np.conj(X))) < 1e-12


def test_inverse_roundtrip():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((4, 8, 24)) + 1j * rng.standard_normal((4, 8, 24))
    y = F.fft3(F.fft3(x), inverse=True)
    assert np.max(np.abs(y - x)) < 1e-13


@pytest.mark.parametrize("n", [192, 256, 384])
def test_library_special_case(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((4, n)) + 1j * rng.standard_normal((4, n))
    assert np.max(np.abs(F.fft(x) - np.fft.fft(x))) < 1e-12 * n
    assert np.max(np.abs(F.fft(x, inverse=True) - np.fft.ifft(x))) < 1e-14 * n


def test_factorize_rejects_other_primes():
    with pytest.raises(ValueError):
        F.factorize(14)
    assert sorted(F.factorize(384)) == sorted([4, 4, 4, 2, 3])
