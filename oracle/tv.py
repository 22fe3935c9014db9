"""Algorithm 3 of the paper (Section 4.4): the TV and l1 + TV problems, with and without
the polarization constraint, FP64, in the printed step order.

Test infrastructure only (see the package docstring).

Problem (Eq. Akiyama_2; Eq. Akiyama without the constraint):
    minimise 1/2 ||Y~ - phi~(S)||_2^2 + iota_U(S) + g(Psi^dagger S) [+ iota_V(Z)
             + iota_E1(S_1, Z_1) + iota_E2(S_2:4, Z_2)]
with phi~ = phi L^-1 and Y~ = Y L^-1 (Stokes-domain data), and
    TV:      g(Psi^dagger S) = sum_i mu_i ||grad S_i||_{2,1},       Psi = grad,
    l1 + TV: g = sum_i nu_i ||S_i||_1 + sum_i mu_i ||grad S_i||_{2,1}, Psi = [Id, grad].

Readings (the paper leaves these open):
  * The gradient grad = [grad_x, grad_y] (Eq. TV) is the forward difference with
    periodic boundaries, like the periodic wavelet transforms of Psi; ||grad||^2 = 8.
  * The "proximity operator of the TV norm" of step 6 acts on the dual variable in
    the range of Psi^dagger = grad, i.e. it is the prox of mu ||.||_{2,1} on gradient
    fields: per pixel, group soft thresholding of the 2-vector (grad_x, grad_y). No
    inner iterations are needed.
  * The data gradient: phi~^dagger(phi~(S) - Y~) = Re(Phi^H (Phi S - Y L^-1)), and
    because L L^H = 2 I this equals 1/2 phi^dagger(phi(S) - Y).
  * Step sizes: the smooth term's gradient is Lipschitz with beta = ||phi~||^2 =
    ||phi||^2 / 2, and tau = 0.99 / (beta / 2 + rho1 ||Psi||^2 [+ rho3]) meets the
    forward-backward primal-dual condition 1/tau - sum rho_i ||K_i||^2 >= beta / 2,
    ||Psi||^2 = 8 (TV) or 9 (l1 + TV: Id stacked on grad). The dual steps are balanced
    against beta, rho1 ||Psi||^2 = rho3 = beta / 2, so that the duals move on the data
    term's scale (with rho = 1 they move ~||phi||^2 times slower than the primal and the
    constraint takes far longer to act).
  * Modes: TV and L1TV carry the constraint (steps 3-12 of Algorithm 3: S with P_U,
    Z, and the epigraph duals C, D as in Algorithm 1); TV_NC and L1TV_NC are the
    problems without it (steps 3, 5, 6 only, S with P_U': Stokes I >= 0).

State: S (4, n, n); Z (2, n, n); A_tv (4, 2, n, n) (x and y components); A_l1
(4, n, n) (l1 + TV only); C (4, n, n); D (2, n, n).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import measurement as meas
from . import prox

TV, TV_NC, L1TV, L1TV_NC = 4, 5, 6, 7
CONSTRAINED = (TV, L1TV)
WITH_L1 = (L1TV, L1TV_NC)


def grad(U: np.ndarray) -> np.ndarray:
    """Forward differences with periodic boundaries: (..., n, n) -> (..., 2, n, n), [d_x, d_y]."""
    gx = np.roll(U, -1, axis=-1) - U        # U[p, q+1] - U[p, q]
    gy = np.roll(U, -1, axis=-2) - U        # U[p+1, q] - U[p, q]
    return np.stack([gx, gy], axis=-3)


def grad_adjoint(G: np.ndarray) -> np.ndarray:
    """grad^T (..., 2, n, n) -> (..., n, n): the transpose of the forward differences."""
    gx, gy = G[..., 0, :, :], G[..., 1, :, :]
    return (np.roll(gx, 1, axis=-1) - gx) + (np.roll(gy, 1, axis=-2) - gy)


def group_soft_threshold(G: np.ndarray, t: np.ndarray) -> np.ndarray:
    """prox of t ||.||_{2,1} on gradient fields (..., 2, n, n): each pixel's 2-vector
    shrunk toward 0 by t (t broadcast over (..., n, n))."""
    norm = np.sqrt(np.sum(G * G, axis=-3, keepdims=True))
    t = np.asarray(t)[..., None, :, :] if np.ndim(t) else t
    scale = np.maximum(0.0, 1.0 - t / np.where(norm > 0, norm, 1.0))
    return G * np.where(norm > 0, scale, 0.0)


def data_gradient(S: np.ndarray, uv: np.ndarray, w: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """phi~^dagger(phi~(S) - Y~) with phi~ = phi L^-1, Y~ = Y L^-1, written through Phi:
    Re(Phi^H (Phi S - Y L^-1)) (S columns are the Stokes maps)."""
    Yt = Y @ np.linalg.inv(meas.L_MIX)
    R = meas.Phi(np.asarray(S, dtype=np.complex128), uv, w) - Yt
    return np.real(meas.Phi_adjoint(R, uv, w, S.shape[-1]))


@dataclasses.dataclass
class TVParams:
    tau: float
    rho1: float
    rho3: float
    mu: np.ndarray            # (4,) TV weights per Stokes map
    nu: np.ndarray            # (4,) l1 weights per Stokes map (l1 + TV only)


def step_sizes(opnorm_sq: float, mode: int, mu, nu=(0.0, 0.0, 0.0, 0.0), rho1: float | None = None,
               rho3: float | None = None, safety: float = 0.99) -> TVParams:
    beta = opnorm_sq / 2.0
    npsi = 9.0 if mode in WITH_L1 else 8.0
    rho1 = beta / (2.0 * npsi) if rho1 is None else rho1
    rho3 = beta / 2.0 if rho3 is None else rho3
    denom = beta / 2.0 + rho1 * npsi
    if mode in CONSTRAINED:
        denom += rho3
    return TVParams(tau=safety / denom, rho1=rho1, rho3=rho3, mu=np.asarray(mu, float), nu=np.asarray(nu, float))


def zero_state(n: int) -> dict:
    return {"S": np.zeros((4, n, n)), "Z": np.zeros((2, n, n)), "Atv": np.zeros((4, 2, n, n)),
            "Al1": np.zeros((4, n, n)), "C": np.zeros((4, n, n)), "D": np.zeros((2, n, n))}


def psi(st: dict, mode: int) -> np.ndarray:
    """Psi A: grad^T A_tv (+ A_l1 for l1 + TV)."""
    out = grad_adjoint(st["Atv"])
    if mode in WITH_L1:
        out = out + st["Al1"]
    return out


def tv_iteration(st: dict, uv: np.ndarray, w: np.ndarray, Y: np.ndarray, p: TVParams, mode: int) -> dict:
    """One iteration of Algorithm 3 in the printed order."""
    S, Z, C, D = st["S"], st["Z"], st["C"], st["D"]
    out = dict(st)
    # Step 3: primal S, gradient step on the data term.
    g = data_gradient(S, uv, w, Y) + psi(st, mode)
    if mode in CONSTRAINED:
        g = g + C
    X = S - p.tau * g
    S1 = prox.proj_U(X) if mode in CONSTRAINED else prox.proj_U_pos(X)
    Sb = 2.0 * S1 - S
    out["S"] = S1
    # Step 4: primal Z.
    if mode in CONSTRAINED:
        Z1 = prox.proj_V(Z - p.tau * D)
        Zb = 2.0 * Z1 - Z
        out["Z"] = Z1
    # Steps 5-6: sparsity duals, A = A~ - rho1 T_{Lambda/rho1}(A~ / rho1).
    At = st["Atv"] + p.rho1 * grad(Sb)
    t = (p.mu / p.rho1)[:, None, None]
    out["Atv"] = At - p.rho1 * group_soft_threshold(At / p.rho1, np.broadcast_to(t, S.shape))
    if mode in WITH_L1:
        Bt = st["Al1"] + p.rho1 * Sb
        out["Al1"] = Bt - p.rho1 * prox.soft_threshold(Bt / p.rho1, np.broadcast_to((p.nu / p.rho1)[:, None, None], S.shape))
    # Steps 7-10: epigraph duals (as Algorithm 1 steps 9-12).
    if mode in CONSTRAINED:
        Ct = C + p.rho3 * Sb
        Dt = D + p.rho3 * Zb
        c1, d1 = prox.proj_E1(Ct[0] / p.rho3, Dt[0] / p.rho3)
        R2, d2 = prox.proj_E2(Ct[1:4] / p.rho3, Dt[1] / p.rho3)
        C1 = np.empty_like(C)
        D1 = np.empty_like(D)
        C1[0] = Ct[0] - p.rho3 * c1
        D1[0] = Dt[0] - p.rho3 * d1
        C1[1:4] = Ct[1:4] - p.rho3 * R2
        D1[1] = Dt[1] - p.rho3 * d2
        out["C"], out["D"] = C1, D1
    return out


def objective(S: np.ndarray, uv: np.ndarray, w: np.ndarray, Y: np.ndarray, p: TVParams, mode: int) -> float:
    """1/2 ||Y~ - phi~(S)||^2 + g(Psi^dagger S) (the indicators are checked separately)."""
    Yt = Y @ np.linalg.inv(meas.L_MIX)
    R = meas.Phi(np.asarray(S, dtype=np.complex128), uv, w) - Yt
    G = grad(S)
    val = 0.5 * float(np.sum(np.abs(R) ** 2)) + float(np.sum(p.mu[:, None, None] * np.sqrt(np.sum(G * G, axis=1))))
    if mode in WITH_L1:
        val += float(np.sum(p.nu[:, None, None] * np.abs(S)))
    return val


def metric_sq(d: dict, p: TVParams, mode: int) -> float:
    """||dz||_M^2, M = [[I/tau, -K^T], [-K, diag(1/rho)]], K: (S, Z) -> (Psi^dagger S, S, Z).
    With the step-size condition the iteration is averaged in this metric, so
    ||z^(k+1) - z^k||_M does not grow."""
    dS = d["S"]
    val = np.sum(dS ** 2) / p.tau + np.sum(d["Atv"] ** 2) / p.rho1
    cross = float(np.sum(grad(dS) * d["Atv"]))
    if mode in WITH_L1:
        val += np.sum(d["Al1"] ** 2) / p.rho1
        cross += float(np.sum(dS * d["Al1"]))
    if mode in CONSTRAINED:
        val += np.sum(d["Z"] ** 2) / p.tau + (np.sum(d["C"] ** 2) + np.sum(d["D"] ** 2)) / p.rho3
        cross += float(np.sum(dS * d["C"]) + np.sum(d["Z"] * d["D"]))
    return float(val - 2.0 * cross)
