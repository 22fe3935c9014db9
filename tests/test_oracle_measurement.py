"""Pins of the oracle's measurement operator phi against facts the mathematics fixes."""
import math

import numpy as np
import pytest

from oracle import measurement as meas
from paper_1801_02417_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def _rand_problem(n=12, M=50, seed=0, omega=2.5):
    rng = np.random.default_rng(seed)
    uv = rng.uniform(-omega, omega, size=(M, 2))
    w = rng.uniform(0.5, 1.5, size=M)
    return rng, uv, w


def test_adjoint_in_real_inner_product():
    """Re<phi S, B> = <S, phi^dagger B> (definition of the adjoint; Stokes maps real, Eq. real_proj)."""
    rng, uv, w = _rand_problem()
    n = 12
    S = rng.normal(size=(4, n, n))
    B = rng.normal(size=(50, 4)) + 1j * rng.normal(size=(50, 4))
    lhs = np.sum(np.real(np.conj(meas.phi(S, uv, w)) * B))
    rhs = np.sum(S * meas.phi_adjoint(B, uv, w, n))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_complex_adjoint_of_Phi():
    """<Phi x, y> = <x, Phi^H y> for complex x, y."""
    rng, uv, w = _rand_problem(seed=1)
    n = 12
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    y = rng.normal(size=50) + 1j * rng.normal(size=50)
    lhs = np.vdot(y, meas.Phi(x, uv, w))
    rhs = np.vdot(meas.Phi_adjoint(y, uv, w, n), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_on_grid_frequencies_match_library_fft():
    """At omega = 2 pi k / n the direct DFT is numpy's FFT up to the centring phase."""
    n = 16
    rng = np.random.default_rng(2)
    x = rng.normal(size=(n, n))
    ky, kx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    uv = np.stack([2 * np.pi * kx.ravel() / n, 2 * np.pi * ky.ravel() / n], axis=1)
    got = meas.Phi(x, uv, np.ones(n * n))
    F = np.fft.fft2(x)                          # sum x[p,q] exp(-2 pi i (ky p + kx q)/n)
    # x = q - n/2, y = p - n/2 adds exp(+i pi (kx + ky)).
    ref = (F * np.exp(1j * np.pi * (kx + ky))).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("stokes,expect", [
    (0, [1, 0, 0, 1]),       # I: RR = LL = I
    (1, [1, 0, 0, -1]),      # Q: RR = Q, LL = -Q
    (2, [0, 1, 1, 0]),       # U: RL = LR = U
    (3, [0, 1j, -1j, 0]),    # V: RL = iV, LR = -iV
])
def test_point_source_at_centre_gives_brightness_vector(stokes, expect):
    """A unit point at the phase centre has flat visibilities S^T L = [I+Q, U+iV, U-iV, I-Q] (Section 2.1)."""
    n = 8
    rng, uv, w = _rand_problem(n=n, M=30, seed=3)
    S = np.zeros((4, n, n))
    S[stokes, n // 2, n // 2] = 1.0
    Y = meas.phi(S, uv, w)
    ref = w[:, None] * np.array(expect)[None, :]
    assert np.max(np.abs(Y - ref)) <= 1e-13


def test_shifted_point_source_phase():
    """A point at (x, y) = (1, -2) gives w exp(-i (omega_u - 2 omega_v)) (the phase convention of Eq. RIME)."""
    n = 8
    rng, uv, w = _rand_problem(n=n, M=20, seed=4)
    S = np.zeros((4, n, n))
    S[0, n // 2 - 2, n // 2 + 1] = 1.0
    Y = meas.phi(S, uv, w)
    ref = w * np.exp(-1j * (uv[:, 0] * 1 - uv[:, 1] * 2))
    assert np.max(np.abs(Y[:, 0] - ref)) <= 1e-13


def test_operator_norm_closed_form_and_power_iteration():
    """L L^H = 2 I, so ||phi||^2 = 2 lambda_max(Re Phi^H Phi); the power iteration must find it."""
    n, M = 5, 18
    rng, uv, w = _rand_problem(n=n, M=M, seed=5, omega=3.0)
    LLh = meas.L_MIX @ np.conj(meas.L_MIX).T
    assert np.allclose(LLh, 2 * np.eye(4), atol=1e-15)
    c = np.arange(n) - n / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")
    Phi = w[:, None] * np.exp(-1j * (np.outer(uv[:, 0], xx.ravel()) + np.outer(uv[:, 1], yy.ravel())))
    lam = np.linalg.eigvalsh(np.real(np.conj(Phi).T @ Phi)).max()
    dense = meas.phi_dense(uv, w, n)
    lam_dense = np.linalg.eigvalsh(dense.T @ dense).max()
    assert abs(lam_dense - 2 * lam) <= 1e-10 * lam_dense
    lam_pow = meas.op_norm_sq(uv, w, n, iters=5000, tol=1e-15)
    assert abs(lam_pow - 2 * lam) <= 1e-8 * lam_pow
    assert abs(meas.op_norm_sq_lanczos(uv, w, n) - 2 * lam) <= 1e-9 * lam


def test_chi2_epsilon_two_sigma_coverage():
    """eps^2 sits 2 std above the chi^2 mean: P(||E|| <= eps) ~ Phi(2) = 0.977 (Section 5.1)."""
    M, sigma = 400, 0.3
    eps = meas.chi2_epsilon(M, sigma)
    hits = 0
    trials = 1500
    for t in range(trials):
        E = inputs.complex_noise(M, sigma, seed=1000 + t)
        hits += np.linalg.norm(E) <= eps
    frac = hits / trials
    assert 0.955 <= frac <= 0.995, frac
    # Mean of ||E||^2 is 8M sigma^2/2 = 4 M sigma^2.
    assert abs(eps ** 2 - (4 * M * sigma ** 2 + 2 * math.sqrt(16 * M) * sigma ** 2 / 2)) < 1e-9


def test_pixel_sampled_adjoint_matches_full_adjoint():
    rng, uv, w = _rand_problem(n=10, M=40, seed=6)
    B = rng.normal(size=(40, 4)) + 1j * rng.normal(size=(40, 4))
    full = meas.phi_adjoint(B, uv, w, 10)
    pix = np.array([[0, 0], [3, 7], [9, 9], [5, 5]])
    got = meas.phi_adjoint_at(B, uv, w, 10, pix)
    assert np.allclose(got, full[:, pix[:, 0], pix[:, 1]], atol=1e-12)


def test_phi_adjoint_grid_equals_the_full_adjoint():
    """The product-grid evaluation of phi^dagger (one matrix product per map) against the full
    adjoint on the same data."""
    rng = np.random.default_rng(21)
    n, M = 16, 300
    uv = rng.uniform(-2.5, 2.5, size=(M, 2))
    w = rng.uniform(0.5, 1.5, size=M)
    B = rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))
    full = meas.phi_adjoint(B, uv, w, n)
    ys, xs = [0, 7, 15], [1, 8, 9, 15]
    got = meas.phi_adjoint_grid(B, uv, w, n, ys, xs)
    assert np.allclose(got, full[:, ys][:, :, xs], rtol=1e-12, atol=1e-10)
