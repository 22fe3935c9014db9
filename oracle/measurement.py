"""Measurement operator phi of Polarized SARA, FP64, as a direct DFT.

Test infrastructure only (see the package docstring).

Data model (Section 2.1, Eq. RIME_disc): Y = phi(S) + E with S in R^{N x 4}
(columns I, Q, U, V) and Y in C^{M x 4}. Without direction-dependent effects
(Section 5.1, Eq. meas_op) phi(S) = Phi S L, where Phi is the Fourier transform
at the sampled frequencies and L is the Stokes-to-brightness mixing of
Section 2.1: S^T L = [I + Q, U + iV, U - iV, I - Q] (correlations RR, RL, LR, LL).

Readings (the paper leaves these open):
  * Pixel (p, q) of an n x n map (row p, column q) sits at centred coordinates
    x = q - n/2, y = p - n/2. Frequencies are given in radians per pixel,
    omega = (omega_u, omega_v), and the phase follows exp(-i 2 pi u.l) of Eq. RIME:
    (Phi s)_m = w_m sum_{p,q} s[p, q] exp(-i (omega_u,m x + omega_v,m y)).
    w_m >= 0 are per-row weights (1 for natural weighting).
  * The oracle evaluates Phi exactly (direct DFT through separable phase
    tables); the paper's G F Z NUFFT factorisation approximates this sum.
  * The adjoint is taken in the real inner product of R^{N x 4}, because the
    Stokes maps are real (P_U = Re, Eq. real_proj): phi^dagger(B) = Re(Phi^H B L^H).
"""
from __future__ import annotations

import math

import numpy as np

# Rows: Stokes I, Q, U, V; columns: correlations RR, RL, LR, LL (Section 2.1).
L_MIX = np.array([[1, 0, 0, 1],
                  [1, 0, 0, -1],
                  [0, 1, 1, 0],
                  [0, 1j, -1j, 0]], dtype=np.complex128)

_CHUNK = 4096


def _phase_tables(uv: np.ndarray, n: int):
    """exp(-i omega_u x) over columns and exp(-i omega_v y) over rows, shapes (M, n)."""
    c = np.arange(n, dtype=np.float64) - n / 2
    eu = np.exp(-1j * np.outer(uv[:, 0], c))
    ev = np.exp(-1j * np.outer(uv[:, 1], c))
    return eu, ev


def _chunk(n: int) -> int:
    return max(64, min(_CHUNK, (1 << 24) // (4 * n)))


def Phi(x: np.ndarray, uv: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Phi applied to a stack of maps x (k, n, n) -> (M, k) complex (Eq. meas_op, direct DFT)."""
    x = np.asarray(x)
    if x.ndim == 2:
        return Phi(x[None], uv, w)[:, 0]
    k, n, _ = x.shape
    M = uv.shape[0]
    out = np.empty((M, k), dtype=np.complex128)
    ch = _chunk(n)
    for m0 in range(0, M, ch):
        m1 = min(M, m0 + ch)
        eu, ev = _phase_tables(uv[m0:m1], n)
        # T[j, p, m] = sum_q x[j, p, q] eu[m, q]  (a matrix product), then sum_p ev[m, p] T[j, p, m].
        T = np.tensordot(x, eu, axes=([2], [1]))
        out[m0:m1] = np.sum(ev.T[None, :, :] * T, axis=1).T * w[m0:m1, None]
    return out


def Phi_adjoint(y: np.ndarray, uv: np.ndarray, w: np.ndarray, n: int) -> np.ndarray:
    """Phi^H applied to columns y (M, k) -> (k, n, n) complex maps."""
    y = np.asarray(y)
    if y.ndim == 1:
        return Phi_adjoint(y[:, None], uv, w, n)[0]
    M, k = y.shape
    out = np.zeros((k, n, n), dtype=np.complex128)
    ch = _chunk(n)
    for m0 in range(0, M, ch):
        m1 = min(M, m0 + ch)
        eu, ev = _phase_tables(uv[m0:m1], n)
        wy = y[m0:m1] * w[m0:m1, None]
        # out[j, p, q] = sum_m conj(ev[m, p]) wy[m, j] conj(eu[m, q])  (a matrix product per j)
        for j in range(k):
            out[j] += np.conj(ev).T @ (wy[:, j:j + 1] * np.conj(eu))
    return out


def phi(S: np.ndarray, uv: np.ndarray, w: np.ndarray) -> np.ndarray:
    """phi(S) = Phi S L (Eq. meas_op): S (4, n, n) real -> (M, 4) complex, columns RR, RL, LR, LL."""
    F = Phi(np.asarray(S, dtype=np.complex128), uv, w)   # (M, 4): Phi I, Phi Q, Phi U, Phi V
    return F @ L_MIX


def phi_adjoint(B: np.ndarray, uv: np.ndarray, w: np.ndarray, n: int) -> np.ndarray:
    """phi^dagger(B) = Re(Phi^H B L^H): (M, 4) complex -> (4, n, n) real maps I, Q, U, V."""
    G = Phi_adjoint(B @ np.conj(L_MIX).T, uv, w, n)      # columns: Stokes I, Q, U, V
    return np.real(G)


def phi_adjoint_at(B: np.ndarray, uv: np.ndarray, w: np.ndarray, n: int, pixels: np.ndarray) -> np.ndarray:
    """phi^dagger(B) at selected pixels only: (4, P) for pixels (P, 2) given as (p, q).

    Direct sum over the rows: Re sum_m exp(+i (omega_u,m x + omega_v,m y)) w_m [B L^H]_{m, s}.
    """
    X = B @ np.conj(L_MIX).T                                   # (M, 4) columns per Stokes map
    out = np.empty((4, len(pixels)))
    for i, (p, q) in enumerate(pixels):
        x, y = q - n / 2, p - n / 2
        e = np.exp(1j * (uv[:, 0] * x + uv[:, 1] * y)) * w
        out[:, i] = np.real(e @ X)
    return out


def phi_adjoint_grid(B: np.ndarray, uv: np.ndarray, w: np.ndarray, n: int, ys, xs) -> np.ndarray:
    """phi^dagger(B) at every pixel (y, x) of the product of the image rows `ys` and columns `xs`:
    (4, len(ys), len(xs)).

    The same sum as phi_adjoint_at, Re sum_m exp(+i (omega_u,m x + omega_v,m y)) w_m [B L^H]_{m,s},
    with the phase split into its y and x factors so that the pixels of the product grid come
    out of one matrix product over the rows m (checks along tile and window boundaries of
    large maps).
    """
    X = (B @ np.conj(L_MIX).T) * w[:, None]                    # (M, 4)
    cy = np.asarray(ys, dtype=np.float64) - n / 2
    cx = np.asarray(xs, dtype=np.float64) - n / 2
    out = np.zeros((4, len(cy), len(cx)))
    M = uv.shape[0]
    ch = 1 << 16
    for m0 in range(0, M, ch):
        m1 = min(M, m0 + ch)
        ex = np.exp(1j * np.outer(uv[m0:m1, 0], cx))            # (m, len(xs))
        ey = np.exp(1j * np.outer(uv[m0:m1, 1], cy))            # (m, len(ys))
        for s in range(4):
            out[s] += np.real((ey * X[m0:m1, s][:, None]).T @ ex)
    return out


def phi_dense(uv: np.ndarray, w: np.ndarray, n: int) -> np.ndarray:
    """Dense real matrix of phi acting on vec(S) (4N reals) -> real/imag parts of vec(Y) (8M).

    Only for tiny problems (operator-norm and adjointness pins).
    """
    N = n * n
    cols = []
    for j in range(4 * N):
        e = np.zeros(4 * N)
        e[j] = 1.0
        y = phi(e.reshape(4, n, n), uv, w)
        cols.append(np.concatenate([y.real.ravel(), y.imag.ravel()]))
    return np.stack(cols, axis=1)


def op_norm_sq(uv: np.ndarray, w: np.ndarray, n: int, iters: int = 200, tol: float = 1e-10,
               seed: int = 0) -> float:
    """||phi||_sp^2 by power iteration on phi^dagger phi (the step-size bound of Section 4.3.3)."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(4, n, n))
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = phi_adjoint(phi(x, uv, w), uv, w, n)
        lam_new = float(np.sum(x * y))
        nrm = np.linalg.norm(y)
        x = y / nrm
        if abs(lam_new - lam) <= tol * abs(lam_new):
            lam = lam_new
            break
        lam = lam_new
    return lam


def op_norm_sq_lanczos(uv: np.ndarray, w: np.ndarray, n: int, tol: float = 1e-12) -> float:
    """||phi||_sp^2 as the largest eigenvalue of phi^dagger phi by Lanczos (scipy eigsh).

    Same quantity as op_norm_sq; Lanczos converges even when the top eigenvalues
    of the PSF-like operator phi^dagger phi are nearly degenerate.
    """
    from scipy.sparse.linalg import LinearOperator, eigsh

    N4 = 4 * n * n

    def mv(v):
        x = np.asarray(v, dtype=np.float64).reshape(4, n, n)
        return phi_adjoint(phi(x, uv, w), uv, w, n).ravel()
    op = LinearOperator((N4, N4), matvec=mv, dtype=np.float64)
    v0 = np.random.default_rng(0).normal(size=N4)
    return float(eigsh(op, k=1, which="LA", tol=tol, v0=v0, return_eigenvectors=False)[0])


def chi2_epsilon(M_b: int, sigma: float) -> float:
    """l2-ball radius of Section 5.1: eps^2 = (8M + 2 sqrt(2 (8M))) sigma^2 / 2.

    The residual norm follows a chi^2 law with 8M real degrees of freedom of
    variance sigma^2/2; the bound sits two standard deviations above its mean.
    """
    dof = 8.0 * M_b
    return math.sqrt((dof + 2.0 * math.sqrt(2.0 * dof)) * sigma * sigma / 2.0)
