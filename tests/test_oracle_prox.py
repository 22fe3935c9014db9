"""Pins of the oracle's projections and prox operators (Section 4.3) against brute force."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import prox


def _brute_projection(x, cons):
    """argmin ||u - x||^2 subject to inequality constraints cons(u) >= 0, by SLSQP from several starts."""
    best = None
    for x0 in (x, np.zeros_like(x), x + 0.1):
        r = minimize(lambda u: np.sum((u - x) ** 2), x0, jac=lambda u: 2 * (u - x),
                     constraints=[{"type": "ineq", "fun": cons}], method="SLSQP",
                     options={"ftol": 1e-15, "maxiter": 500})
        if best is None or r.fun < best.fun:
            best = r
    return best.x


def test_proj_V_brute_force_and_idempotence():
    rng = np.random.default_rng(0)
    for _ in range(40):
        z = rng.normal(size=2) * 2
        got = prox.proj_V(z.reshape(2, 1))[:, 0]
        ref = _brute_projection(z, lambda u: -(u[0] + u[1]))
        assert np.allclose(got, ref, atol=1e-6)
        assert np.allclose(prox.proj_V(got.reshape(2, 1))[:, 0], got, atol=1e-15)


def test_proj_E1_brute_force_and_moreau():
    rng = np.random.default_rng(1)
    for _ in range(40):
        c, d = rng.normal(size=2) * 2
        pc, pd_ = prox.proj_E1(np.array([c]), np.array([d]))
        ref = _brute_projection(np.array([c, d]), lambda u: u[0] + u[1])   # -c <= d
        assert np.allclose([pc[0], pd_[0]], ref, atol=1e-6)
        # Moreau for a cone K: x = P_K x + P_{K polar} x with orthogonal parts.
        r = np.array([c - pc[0], d - pd_[0]])
        assert abs(r @ np.array([pc[0], pd_[0]])) < 1e-12
        assert r[0] <= 1e-15 and abs(r[0] - r[1]) < 1e-12    # polar cone: t(-1, -1), t >= 0


def test_proj_E2_brute_force_and_moreau():
    rng = np.random.default_rng(2)
    cases = [rng.normal(size=4) * 2 for _ in range(60)]
    cases += [np.array([0.0, 0.0, 0.0, -1.0]), np.array([0.0, 0.0, 0.0, 2.0]),
              np.array([3.0, 0.0, 0.0, -3.0]), np.array([1.0, 1.0, 1.0, np.sqrt(3.0)])]
    for v in cases:
        R = v[:3].reshape(3, 1)
        d = np.array([v[3]])
        pR, pdd = prox.proj_E2(R, d)
        got = np.concatenate([pR[:, 0], pdd])
        ref = _brute_projection(v, lambda u: u[3] - np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2 + 1e-300))
        assert np.allclose(got, ref, atol=2e-5), (v, got, ref)   # SLSQP is approximate at the apex
        assert np.linalg.norm(got[:3]) <= got[3] + 1e-12
        r = v - got
        assert abs(r @ got) < 1e-10
        assert np.linalg.norm(r[:3]) <= -r[3] + 1e-10          # polar cone of the SOC is -SOC
        pR2, pd2 = prox.proj_E2(pR, pdd)
        assert np.allclose(np.concatenate([pR2[:, 0], pd2]), got, atol=1e-14)


def test_proj_P_brute_force_and_moreau():
    """The polarization set P (Eq. pol_const) is the second-order cone {I >= ||(Q, U, V)||}."""
    rng = np.random.default_rng(5)
    cases = [rng.normal(size=4) * 2 for _ in range(60)]
    cases += [np.array([-1.0, 0.0, 0.0, 0.0]), np.array([2.0, 0.0, 0.0, 0.0]),
              np.array([-3.0, 3.0, 0.0, 0.0]), np.array([np.sqrt(3.0), 1.0, 1.0, 1.0]),
              np.array([1.0, 0.3, -0.2, 0.1])]
    for v in cases:
        got = prox.proj_P(v.reshape(4, 1))[:, 0]
        ref = _brute_projection(v, lambda u: u[0] - np.sqrt(u[1] ** 2 + u[2] ** 2 + u[3] ** 2 + 1e-300))
        assert np.allclose(got, ref, atol=2e-5), (v, got, ref)
        assert np.linalg.norm(got[1:]) <= got[0] + 1e-12
        if np.linalg.norm(v[1:]) <= v[0]:
            assert np.array_equal(got, v)                       # points of P are kept
        r = v - got
        assert abs(r @ got) < 1e-10                             # Moreau: orthogonal parts
        assert np.linalg.norm(r[1:]) <= -r[0] + 1e-10           # r in the polar cone -P
        assert np.allclose(prox.proj_P(got.reshape(4, 1))[:, 0], got, atol=1e-14)


def test_soft_threshold_is_prox_and_clamp_identity():
    """T is the prox of t|.| (1D brute force), and A - rho T_{T/rho}(A/rho) = clamp(A, -T, T)."""
    rng = np.random.default_rng(3)
    grid = np.linspace(-10, 10, 400001)
    for _ in range(20):
        a, t = rng.normal() * 3, abs(rng.normal())
        got = prox.soft_threshold(np.array([a]), np.array([t]))[0]
        ref = grid[np.argmin(t * np.abs(grid) + 0.5 * (grid - a) ** 2)]
        assert abs(got - ref) < 1e-4
    A = rng.normal(size=1000) * 3
    T = np.abs(rng.normal(size=1000))
    rho = 0.7
    lhs = A - rho * prox.soft_threshold(A / rho, T / rho)
    assert np.allclose(lhs, np.clip(A, -T, T), atol=1e-14)


def test_ball_projection_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(20):
        Y = rng.normal(size=3) + 1j * rng.normal(size=3)
        X = Y + 2 * (rng.normal(size=3) + 1j * rng.normal(size=3))
        radius = abs(rng.normal()) + 0.1
        got = prox.proj_ball(X, Y, radius)
        xr = np.concatenate([X.real, X.imag])
        yr = np.concatenate([Y.real, Y.imag])
        ref = _brute_projection(xr, lambda u: radius ** 2 - np.sum((u - yr) ** 2))
        assert np.allclose(np.concatenate([got.real, got.imag]), ref, atol=1e-6)
        assert np.allclose(prox.proj_ball(got, Y, radius), got, atol=1e-14)


def test_positivity_projection():
    X = np.array([[-1.0, 2.0], [-3.0, 4.0], [5.0, -6.0], [-7.0, 8.0]])
    out = prox.proj_U_pos(X)
    assert np.array_equal(out[0], [0.0, 2.0])
    assert np.array_equal(out[1:], X[1:])
