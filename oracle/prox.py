"""Projections and proximity operators of Polarized SARA (Section 4.3), FP64.

Test infrastructure only (see the package docstring).

Readings:
  * Soft threshold (Eq. soft_thresh): the printed first case, -A + gamma W / rho1
    for A < -gamma W / rho1, is a sign typo; the proximity operator of the
    weighted l1 norm is the standard soft threshold, A + gamma W / rho1 there.
  * Tie cases: P_E1 keeps (c, d) when c + d >= 0 (Eq. proj_e1); P_E2 uses the
    strict inequalities of Eq. proj_e2_def. Both forms are continuous across the
    boundaries. For ||r|| = 0 and d <= 0 the projection is (0, 0).
"""
from __future__ import annotations

import numpy as np


def proj_U(X: np.ndarray) -> np.ndarray:
    """P_U = Re (Eq. real_proj)."""
    return np.real(X)


def proj_U_pos(X: np.ndarray) -> np.ndarray:
    """P_U' (Eq. pos_set, Section 5.2): real part, with Stokes I (row 0) clipped at 0."""
    out = np.array(np.real(X), copy=True)
    out[0] = np.maximum(out[0], 0.0)
    return out


def proj_V(Z: np.ndarray) -> np.ndarray:
    """P_V onto {z1 + z2 <= 0} per pixel (Section 4.3.1, after Eq. set_V). Z: (2, ...)."""
    z1, z2 = Z[0], Z[1]
    keep = z1 + z2 <= 0
    return np.stack([np.where(keep, z1, 0.5 * (z1 - z2)),
                     np.where(keep, z2, 0.5 * (z2 - z1))])


def proj_E1(c: np.ndarray, d: np.ndarray):
    """P_E1, epigraph of h1(s) = -s, per pixel (Eq. proj_e1)."""
    keep = c + d >= 0
    return np.where(keep, c, 0.5 * (c - d)), np.where(keep, d, 0.5 * (d - c))


def proj_E2(R: np.ndarray, d: np.ndarray):
    """P_E2, epigraph of h2(r) = ||r||_2 in R^3, per pixel (Eq. proj_e2_def). R: (3, ...)."""
    nr = np.sqrt(np.sum(R * R, axis=0))
    inside = nr < d
    zero = nr < -d
    safe = np.where(nr > 0, nr, 1.0)
    alpha = 0.5 * (1.0 + d / safe)
    Rp = np.where(zero, 0.0, np.where(inside, R, alpha * R))
    dp = np.where(zero, 0.0, np.where(inside, d, alpha * nr))
    # ||r|| = 0 with d <= 0: the projection onto the cone is the apex.
    apex = (nr == 0) & (d <= 0)
    Rp = np.where(apex, 0.0, Rp)
    dp = np.where(apex, 0.0, dp)
    return Rp, dp


def proj_P(S: np.ndarray) -> np.ndarray:
    """Projection onto the polarization set P = {sqrt(Q^2 + U^2 + V^2) <= I} per pixel (Eq. pol_const).

    P is the second-order cone in which Stokes I plays the role of the epigraph
    variable of h2(r) = ||r||_2 over r = (Q, U, V), i.e. E2 with d = I, so its
    projection is the closed form of Eq. proj_e2_def applied to (r, d) = (S_2:4, S_1).
    S: (4, ...); returns the projected (I, Q, U, V).
    """
    R, d = proj_E2(S[1:4], S[0])
    return np.concatenate([d[None], R])


def soft_threshold(A: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Component-wise prox of the weighted l1 norm with thresholds T >= 0 (Eq. soft_thresh, sign typo fixed)."""
    return np.where(A < -T, A + T, np.where(A > T, A - T, 0.0))


def proj_ball(X: np.ndarray, Y: np.ndarray, radius: float) -> np.ndarray:
    """Projection onto the l2 ball B(Y, radius) (Section 4.3.2, data fidelity)."""
    r = X - Y
    nr = np.sqrt(np.sum(np.abs(r) ** 2))
    if nr > radius:
        return Y + radius * r / nr
    return X
