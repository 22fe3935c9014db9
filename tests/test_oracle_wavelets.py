"""Pins of the oracle's SARA dictionary (Section 4.1) against wavelet theory."""
import math

import numpy as np
import pytest

from oracle import wavelets as wav


@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_filter_defining_identities(p):
    """Length 2p, sum sqrt 2, double-shift orthonormal, p vanishing moments, extremal phase."""
    h = wav.FILTERS[p]
    g = wav.highpass(h)
    assert len(h) == 2 * p
    assert abs(h.sum() - math.sqrt(2)) < 1e-13
    for k in range(p):
        dot = float(np.dot(h[2 * k:], h[:len(h) - 2 * k]))
        assert abs(dot - (1.0 if k == 0 else 0.0)) < 1e-12
    j = np.arange(2 * p, dtype=np.float64)
    for k in range(p):
        assert abs(np.sum(g * j ** k)) < 1e-9 * max(1.0, float(np.sum(np.abs(g) * j ** k)))
    # Extremal phase: apart from the p-fold zero at z = -1, every zero of
    # sum_j h[j] z^(2p-1-j) lies inside the unit circle.
    # Divide out (1 + z)^p (a p-fold root is too ill-conditioned for np.roots).
    q = h.copy()
    for _ in range(p):
        q, rem = np.polydiv(q, [1.0, 1.0])
        assert np.max(np.abs(rem)) < 1e-12
    if len(q) > 1:
        assert np.all(np.abs(np.roots(q)) < 1.0)


def test_db1_is_haar_and_db2_closed_form():
    assert np.allclose(wav.FILTERS[1], [1 / math.sqrt(2)] * 2, atol=1e-15)
    s3 = math.sqrt(3)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2))
    assert np.allclose(wav.FILTERS[2], ref, atol=1e-14)


def test_haar_one_level_2d_closed_form():
    """One Haar level on a 2x2 block: sums and differences over sqrt(2)^2."""
    x = np.array([[1.0, 2.0], [3.0, 5.0]])
    c = wav.dwt2(x, wav.FILTERS[1], 1)
    a, b, cc, d = 1.0, 2.0, 3.0, 5.0
    assert np.isclose(c[0, 0], (a + b + cc + d) / 2)
    assert np.isclose(c[0, 1], (a - b + cc - d) / 2)     # x-high, y-low
    assert np.isclose(c[1, 0], (a + b - cc - d) / 2)     # x-low, y-high
    assert np.isclose(c[1, 1], (a - b - cc + d) / 2)


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_analysis_matches_fft_circular_correlation(p):
    """One periodic level equals an FFT-computed circular correlation, then keep even indices."""
    rng = np.random.default_rng(p)
    n = 32
    x = rng.normal(size=n)
    h = wav.FILTERS[p]
    g = wav.highpass(h)

    def corr(f):
        fp = np.zeros(n)
        for j, v in enumerate(f):
            fp[j % n] += v
        return np.real(np.fft.ifft(np.fft.fft(x) * np.conj(np.fft.fft(fp))))[::2]
    lo, hi = wav.analysis_1d(x, h, axis=0)
    assert np.allclose(lo, corr(h), atol=1e-12)
    assert np.allclose(hi, corr(g), atol=1e-12)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("n,levels", [(16, 3), (64, 4), (8, 3)])
def test_perfect_reconstruction_and_parseval(p, n, levels):
    rng = np.random.default_rng(10 * p + n)
    x = rng.normal(size=(n, n))
    c = wav.dwt2(x, wav.FILTERS[p], levels)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(wav.idwt2(c, wav.FILTERS[p], levels) - x)) < 1e-12


def test_multilevel_haar_pyramid():
    """L Haar levels: the coarsest coefficient of a constant map is mean * n (orthonormal scaling)."""
    n = 16
    x = np.full((n, n), 3.0)
    c = wav.dwt2(x, wav.FILTERS[1], 4)
    assert abs(c[0, 0] - 3.0 * n) < 1e-12
    assert np.max(np.abs(c.ravel()[1:])) < 1e-12


def test_psi_tight_frame_and_adjoint():
    """Psi Psi^dagger = Id, ||Psi^dagger x|| = ||x||, <Psi^dagger x, a> = <x, Psi a>."""
    rng = np.random.default_rng(7)
    n, L = 32, 3
    x = rng.normal(size=(4, n, n))
    a = rng.normal(size=(4, 9, n, n))
    c = wav.psi_adjoint(x, L)
    assert c.shape == (4, 9, n, n)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(wav.psi(c, L) - x)) < 1e-12
    lhs = float(np.sum(c * a))
    rhs = float(np.sum(x * wav.psi(a, L)))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_level_shift_equivariance():
    """Shifting the map by 2^L pixels circularly shifts every subband by 2^(L-l) at level l."""
    rng = np.random.default_rng(8)
    n, L = 32, 3
    x = rng.normal(size=(n, n))
    h = wav.FILTERS[4]
    c0 = wav.dwt2(x, h, L)
    c1 = wav.dwt2(np.roll(x, (1 << L, 0), axis=(1, 0)), h, L)
    m = n
    for lev in range(1, L + 1):
        k = m // 2
        s = (1 << L) >> lev
        assert np.allclose(np.roll(c0[:k, k:m], s, axis=1), c1[:k, k:m], atol=1e-12)
        m = k
