"""Algorithms 1 and 2 of Polarized SARA (Section 4.3), FP64, in the paper's step order.

Test infrastructure only (see the package docstring).

State: S (4, n, n) Stokes maps I, Q, U, V; Z (2, n, n) epigraph auxiliary;
A (4, 9, n, n) dual of the l1 term; B (M, 4) complex dual of the data term;
C (4, n, n) and D (2, n, n) duals of the epigraph constraints. T = gamma W
(4, 9, n, n) are the soft-threshold sizes.

Readings (the paper leaves these open or prints them inconsistently):
  * l2 ball radius: step 8 prints P_{B(Y, eps/rho2)}(B~/rho2). The Moreau identity
    for the conjugate of the indicator of B(Y, eps) (Eq. f_diff) gives radius eps,
    which is also the radius the stopping rule checks, so radius eps is used;
    ``literal_ball=True`` selects the printed radius eps/rho2 instead.
  * Several data blocks: f is the sum of the indicators of per-block balls
    B(Y_b, eps_b); its prox acts block by block (one block is the paper's case).
  * Step sizes (Section 4.3.3 gives only 1/tau - rho1 ||Psi||^2 - rho2 ||phi||^2
    - rho3 >= 0): rho1 = rho3 = 1, rho2 = 1/||phi||^2, ||Psi|| = 1 (tight frame),
    tau = 0.99 / (sum of the rho_i ||K_i||^2 of the terms present in the mode).
  * Modes: POLARIZED is Algorithm 1 in full. NO_CONSTRAINT (Section 5.2) updates
    S, A, B only with P_U' (Stokes I >= 0). NNLS (Section 4.3.4, initialisation)
    updates S and B only, with P_U' and g = 0; every other variable stays zero.
    SOC is not in the paper: the same problem as POLARIZED, with the polarization
    constraint iota_P(S) (Eq. pol_const) given its own dual C under the identity
    operator instead of the epigraphical split of Section 4.3.1. Step 3 is
    unchanged, step 4 and Z, D drop out, and steps 9-12 become
    C = C~ - rho3 P_P(C~ / rho3), C~ = C + rho3 (2 S^(k+1) - S^(k)), with the
    closed-form cone projection P_P (prox.proj_P). tau uses the same sum
    rho1 + rho2 ||phi||^2 + rho3 (||Id|| = 1).
  * N_p (Section 5.2) uses all of S_{n,2:4}; the threshold zeta is
    ``zeta_sigma`` times the rms of the Stokes I residual image phi^dagger(Y - phi S)
    in units of its PSF peak 2 sum w_m^2.
  * A reweight count r with k iterations: r + 1 cycles of k // (r + 1) iterations,
    the first in NNLS mode, each later one preceded by a reweight
    (Algorithm 2). delta^(1) = 0.1 max |Psi^dagger S_nnls|, halved at each reweight.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import measurement as meas
from . import prox
from . import wavelets as wav

POLARIZED, NO_CONSTRAINT, NNLS, SOC = 0, 1, 2, 3


@dataclasses.dataclass
class Problem:
    n: int
    levels: int
    uv: np.ndarray          # (M, 2) rad/pixel
    w: np.ndarray           # (M,)
    Y: np.ndarray           # (M, 4) complex
    offsets: np.ndarray     # (nblocks + 1,)
    eps: np.ndarray         # (nblocks,)


@dataclasses.dataclass
class Params:
    tau: float
    rho1: float
    rho2: float
    rho3: float
    literal_ball: bool = False


def step_sizes(opnorm_sq: float, mode: int, rho1: float = 1.0, rho3: float = 1.0,
               rho2: float | None = None, safety: float = 0.99) -> Params:
    """Step sizes meeting the condition of Section 4.3.3 with ||Psi|| = 1."""
    if rho2 is None:
        rho2 = 1.0 / opnorm_sq
    denom = rho2 * opnorm_sq
    if mode in (POLARIZED, NO_CONSTRAINT, SOC):
        denom += rho1
    if mode in (POLARIZED, SOC):
        denom += rho3
    return Params(tau=safety / denom, rho1=rho1, rho2=rho2, rho3=rho3)


def zero_state(n: int, M: int) -> dict:
    return {"S": np.zeros((4, n, n)), "Z": np.zeros((2, n, n)), "A": np.zeros((4, 9, n, n)),
            "B": np.zeros((M, 4), dtype=np.complex128), "C": np.zeros((4, n, n)),
            "D": np.zeros((2, n, n))}


def ball_step(Bt: np.ndarray, prob: Problem, p: Params) -> np.ndarray:
    """Algorithm 1 step 8 per block: B = B~ - rho2 P_B(Y_b, eps_b)(B~ / rho2)."""
    out = np.empty_like(Bt)
    for b in range(len(prob.eps)):
        sl = slice(int(prob.offsets[b]), int(prob.offsets[b + 1]))
        radius = prob.eps[b] / p.rho2 if p.literal_ball else prob.eps[b]
        out[sl] = Bt[sl] - p.rho2 * prox.proj_ball(Bt[sl] / p.rho2, prob.Y[sl], radius)
    return out


def pd_iteration(st: dict, prob: Problem, T: np.ndarray, p: Params, mode: int = POLARIZED) -> dict:
    """One iteration of Algorithm 1 (steps 3-12) in the printed order."""
    S, Z, A, B, C, D = st["S"], st["Z"], st["A"], st["B"], st["C"], st["D"]
    n, L = prob.n, prob.levels
    # Step 3: primal S.
    grad = meas.phi_adjoint(B, prob.uv, prob.w, n)
    if mode != NNLS:
        grad = grad + wav.psi(A, L)
    if mode in (POLARIZED, SOC):
        grad = grad + C
    X = S - p.tau * grad
    S1 = prox.proj_U(X) if mode in (POLARIZED, SOC) else prox.proj_U_pos(X)
    Sb = 2.0 * S1 - S
    out = dict(st)
    out["S"] = S1
    # Step 4: primal Z.
    if mode == POLARIZED:
        Z1 = prox.proj_V(Z - p.tau * D)
        Zb = 2.0 * Z1 - Z
        out["Z"] = Z1
    # Steps 5-6: sparsity dual.
    if mode != NNLS:
        At = A + p.rho1 * wav.psi_adjoint(Sb, L)
        out["A"] = At - p.rho1 * prox.soft_threshold(At / p.rho1, T / p.rho1)
    # Steps 7-8: data-fidelity dual.
    Bt = B + p.rho2 * meas.phi(Sb, prob.uv, prob.w)
    out["B"] = ball_step(Bt, prob, p)
    # Steps 9-12: epigraph duals.
    if mode == POLARIZED:
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
    if mode == SOC:
        Ct = C + p.rho3 * Sb
        out["C"] = Ct - p.rho3 * prox.proj_P(Ct / p.rho3)
    return out


def reweight(S: np.ndarray, levels: int, delta: float) -> np.ndarray:
    """Weights of Eq. weights: W_ji = delta / (delta + |[Psi^dagger S]_ji|), shape (4, 9, n, n)."""
    c = np.abs(wav.psi_adjoint(S, levels))
    return delta / (delta + c)


def residual_norms(S: np.ndarray, prob: Problem) -> np.ndarray:
    """Per-block ||phi(S) - Y||_2 (stopping rule of Section 5.5)."""
    r = meas.phi(S, prob.uv, prob.w) - prob.Y
    return np.array([math.sqrt(float(np.sum(np.abs(r[int(prob.offsets[b]):int(prob.offsets[b + 1])]) ** 2)))
                     for b in range(len(prob.eps))])


def relative_change(S_new: np.ndarray, S_old: np.ndarray) -> np.ndarray:
    """Per-map ||S_i^(k+1) - S_i^(k)|| / ||S_i^(k)|| (Eq. stop_crit).

    Where ||S_i^(k)|| = 0: 0 if the map stays zero (V in the paper's data), inf if it moves.
    """
    num = np.sqrt(np.sum((S_new - S_old) ** 2, axis=(1, 2)))
    den = np.sqrt(np.sum(S_old ** 2, axis=(1, 2)))
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))


def violation_count(S: np.ndarray, zeta: float) -> int:
    """Pixels of the polarization error image p (Section 5.2) above zeta: -I + ||(Q,U,V)|| > zeta."""
    pv = -S[0] + np.sqrt(S[1] ** 2 + S[2] ** 2 + S[3] ** 2)
    return int(np.count_nonzero(pv > zeta))


def stop_rule(S_new: np.ndarray, S_old: np.ndarray, prob: Problem, rel_tol: float = 1e-5,
              resid_tol: float = 5e-3, np_tol: float = 0.5, zeta_sigma: float = 3.0,
              constrained: bool = True, maps: int = 4) -> dict:
    """The stopping rule of Section 5.5 after the iteration S_old -> S_new.

    rel: max over the first `maps` maps of the relative change (Eq. stop_crit) <= rel_tol;
    the paper takes i = 1..3 (I, Q, U: its V is zero); maps = 4 takes V as well (a map that
    stays zero contributes 0). resid: ||phi(S) - Y||_b <= (1 + vartheta) eps_b for every
    block. np: with the polarization constraint, N_p = 100 * (pixels above zeta) / N <= varrho
    (percent, Section 5.2). converged: all three.
    """
    rel = bool(np.max(relative_change(S_new, S_old)[:maps]) <= rel_tol)
    resid = bool(np.all(residual_norms(S_new, prob) <= (1.0 + resid_tol) * prob.eps))
    n_p = 100.0 * violation_count(S_new, zeta_threshold(S_new, prob, zeta_sigma)) / S_new[0].size
    np_ok = (not constrained) or n_p <= np_tol
    return {"rel": rel, "resid": resid, "np": np_ok, "N_p": n_p, "converged": rel and resid and np_ok}


def zeta_threshold(S: np.ndarray, prob: Problem, zeta_sigma: float = 3.0) -> float:
    """zeta = zeta_sigma * rms(residual Stokes I image) / PSF peak (reading of Section 5.2)."""
    r = prob.Y - meas.phi(S, prob.uv, prob.w)
    img = meas.phi_adjoint(r, prob.uv, prob.w, prob.n)[0]
    psf_peak = 2.0 * float(np.sum(prob.w ** 2))
    return zeta_sigma * math.sqrt(float(np.mean(img ** 2))) / psf_peak


def metric_sq(dS, dZ, dA, dB, dC, dD, prob: Problem, p: Params, mode: int) -> float:
    """||dz||_M^2 for the primal-dual metric M = [[I/tau, -K^T], [-K, diag(1/rho)]].

    K maps (S, Z) to (Psi^dagger S, phi(S), S, Z) (SOC: (Psi^dagger S, phi(S), S)). Algorithm 1 is a proximal point
    step in this metric, so ||z^(k+1) - z^k||_M is non-increasing when the step-size
    condition of Section 4.3.3 holds.
    """
    val = (np.sum(dS ** 2) + (np.sum(dZ ** 2) if mode == POLARIZED else 0.0)) / p.tau
    cross = float(np.sum(np.real(np.conj(meas.phi(dS, prob.uv, prob.w)) * dB)))
    val += np.sum(np.abs(dB) ** 2) / p.rho2
    if mode != NNLS:
        val += np.sum(dA ** 2) / p.rho1
        cross += float(np.sum(wav.psi_adjoint(dS, prob.levels) * dA))
    if mode == POLARIZED:
        val += (np.sum(dC ** 2) + np.sum(dD ** 2)) / p.rho3
        cross += float(np.sum(dS * dC) + np.sum(dZ * dD))
    if mode == SOC:
        val += np.sum(dC ** 2) / p.rho3
        cross += float(np.sum(dS * dC))
    return float(val - 2.0 * cross)


def run(st: dict, prob: Problem, T: np.ndarray, p: Params, iters: int, mode: int = POLARIZED) -> dict:
    for _ in range(iters):
        st = pd_iteration(st, prob, T, p, mode)
    return st


def solve(prob: Problem, iterations: int, reweights: int, gamma: float, opnorm_sq: float,
          delta_factor: float = 0.1, delta_decay: float = 0.5, mode: int = POLARIZED) -> dict:
    """Algorithm 2 with the NNLS start (Section 4.3.4): fixed iteration budget; the reweighted
    cycles run in `mode` (POLARIZED, or SOC for the direct cone dual)."""
    n, M = prob.n, prob.Y.shape[0]
    cycles = reweights + 1
    per = iterations // cycles
    st = zero_state(n, M)
    T = np.zeros((4, 9, n, n))
    st = run(st, prob, T, step_sizes(opnorm_sq, NNLS), per, NNLS)
    delta = delta_factor * float(np.max(np.abs(wav.psi_adjoint(st["S"], prob.levels))))
    p = step_sizes(opnorm_sq, mode)
    for _ in range(reweights):
        T = gamma * reweight(st["S"], prob.levels, delta)
        st = run(st, prob, T, p, per, mode)
        delta *= delta_decay
    return st
