"""SARA dictionary Psi (Section 4.1), FP64: Dirac plus Daubechies db1..db8.

Test infrastructure only (see the package docstring).

Readings (the paper names the bases only):
  * Each Daubechies basis is the orthonormal, periodic (circular boundary),
    separable 2D Mallat transform with ``levels`` levels. Periodic boundaries keep
    every basis orthonormal with exactly N coefficients, so J = 9N.
  * The concatenation is scaled by 1/sqrt(9) = 1/3, making Psi a tight frame:
    Psi Psi^dagger = Id and ||Psi||_sp = 1.
  * Filters are the extremal-phase Daubechies scaling filters with p vanishing
    moments, length 2p (Daubechies 1988), built here by spectral factorisation.
  * One analysis level of a length-n signal x (n even), low- and high-pass:
        a[k] = sum_j h[j] x[(2k + j) mod n],   d[k] = sum_j g[j] x[(2k + j) mod n],
    with g[j] = (-1)^j h[2p - 1 - j].  Synthesis is the transpose.
  * 2D level: filter along columns (axis 1) into halves [low | high], then along
    rows (axis 0) into [low ; high]. The n x n Mallat layout holds
    [0:h, 0:h] approximation (recursed), [0:h, h:n] x-high/y-low,
    [h:n, 0:h] x-low/y-high, [h:n, h:n] x-high/y-high, with h = n/2.
  * Coefficient array of one map: (9, n, n), basis 0 = Dirac, b = db_b for b=1..8.
"""
from __future__ import annotations

import math

import numpy as np

N_BASES = 9
PSI_SCALE = 1.0 / 3.0


def daubechies_filter(p: int) -> np.ndarray:
    """Scaling filter h of the Daubechies wavelet with p vanishing moments (length 2p).

    |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)) with P(y) = sum_{k<p} C(p-1+k, k) y^k.
    Each root y_k of P gives z-roots of (2 - z - 1/z)/4 = y_k; the root inside the
    unit circle is kept (extremal phase). Then
    h(z) = c (1 + z)^p prod_k (z - z_k), with c fixing sum(h) = sqrt(2).
    """
    if p == 1:
        return np.array([1.0, 1.0]) / math.sqrt(2.0)
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]       # P(y), ascending powers
    yroots = np.roots(coeffs[::-1])
    zroots = []
    for yk in yroots:
        # z^2 - (2 - 4 y) z + 1 = 0
        b = 2.0 - 4.0 * yk
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
        zroots.append(z1 if abs(z1) < 1.0 else z2)
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    for zk in zroots:
        poly = np.convolve(poly, [1.0, -zk])
    # np.convolve builds the coefficients in descending powers of z; that order is
    # the usual one for the scaling filter (db2: h[0] = (1 + sqrt 3) / (4 sqrt 2)).
    h = np.real(poly)
    return h * (math.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    """Alternating flip g[j] = (-1)^j h[L-1-j]."""
    Lf = len(h)
    return np.array([(-1) ** j * h[Lf - 1 - j] for j in range(Lf)])


FILTERS = {b: daubechies_filter(b) for b in range(1, 9)}


def analysis_1d(x: np.ndarray, h: np.ndarray, axis: int):
    """One periodic analysis level along ``axis``: returns (low, high), each half length."""
    g = highpass(h)
    n = x.shape[axis]
    k = np.arange(n // 2)[:, None]
    j = np.arange(len(h))[None, :]
    xt = np.take(np.moveaxis(x, axis, -1), (2 * k + j) % n, axis=-1)   # [..., k, j] = x[(2k + j) mod n]
    return np.moveaxis(xt @ h, -1, axis), np.moveaxis(xt @ g, -1, axis)


def synthesis_1d(lo: np.ndarray, hi: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of analysis_1d: x[i] = sum_k lo[k] h[i-2k] + hi[k] g[i-2k] (indices mod n)."""
    g = highpass(h)
    lo = np.moveaxis(lo, axis, -1)
    hi = np.moveaxis(hi, axis, -1)
    n = 2 * lo.shape[-1]
    ul = np.zeros(lo.shape[:-1] + (n,))
    uh = np.zeros(lo.shape[:-1] + (n,))
    ul[..., 0::2] = lo                                                  # upsample by 2
    uh[..., 0::2] = hi
    i = np.arange(n)[:, None]
    j = np.arange(len(h))[None, :]
    idx = (i - j) % n                                                   # x[i] = sum_j h[j] u[i - j]
    x = np.take(ul, idx, axis=-1) @ h + np.take(uh, idx, axis=-1) @ g
    return np.moveaxis(x, -1, axis)


def dwt2(x: np.ndarray, h: np.ndarray, levels: int) -> np.ndarray:
    """Multilevel periodic 2D analysis of an n x n map into the Mallat layout."""
    out = np.array(x, dtype=np.float64, copy=True)
    m = out.shape[0]
    for _ in range(levels):
        blk = out[:m, :m]
        lo, hi = analysis_1d(blk, h, axis=1)
        ll, lh = analysis_1d(lo, h, axis=0)
        hl, hh = analysis_1d(hi, h, axis=0)
        k = m // 2
        out[:k, :k] = ll
        out[:k, k:m] = hl        # x-high, y-low
        out[k:m, :k] = lh        # x-low, y-high
        out[k:m, k:m] = hh
        m = k
    return out


def idwt2(c: np.ndarray, h: np.ndarray, levels: int) -> np.ndarray:
    """Inverse (transpose) of dwt2."""
    out = np.array(c, dtype=np.float64, copy=True)
    n = out.shape[0]
    m = n >> (levels - 1)
    for _ in range(levels):
        k = m // 2
        ll, hl = out[:k, :k], out[:k, k:m]
        lh, hh = out[k:m, :k], out[k:m, k:m]
        lo = synthesis_1d(ll, lh, h, axis=0)
        hi = synthesis_1d(hl, hh, h, axis=0)
        out[:m, :m] = synthesis_1d(lo, hi, h, axis=1)
        m *= 2
    return out


def check_levels(n: int, levels: int) -> None:
    if n % (1 << levels) != 0 or levels < 1:
        raise ValueError(f"n={n} must be divisible by 2^levels={1 << levels}")


def psi_adjoint(S: np.ndarray, levels: int) -> np.ndarray:
    """Analysis Psi^dagger: maps (k, n, n) -> coefficients (k, 9, n, n), tight-frame scaled."""
    S = np.asarray(S, dtype=np.float64)
    k, n, _ = S.shape
    check_levels(n, levels)
    out = np.empty((k, N_BASES, n, n))
    for i in range(k):
        out[i, 0] = S[i]
        for b in range(1, 9):
            out[i, b] = dwt2(S[i], FILTERS[b], levels)
    return PSI_SCALE * out


def psi(A: np.ndarray, levels: int) -> np.ndarray:
    """Synthesis Psi: coefficients (k, 9, n, n) -> maps (k, n, n)."""
    A = np.asarray(A, dtype=np.float64)
    k, nb, n, _ = A.shape
    out = np.empty((k, n, n))
    for i in range(k):
        acc = A[i, 0].copy()
        for b in range(1, 9):
            acc += idwt2(A[i, b], FILTERS[b], levels)
        out[i] = acc
    return PSI_SCALE * out
