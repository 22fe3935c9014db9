"""Pins of the FP64 oracle for Algorithm 3 (TV and l1 + TV problems), on CPU: the
gradient operator against its closed forms, the dual step against a brute-force prox and
the Moreau identity, the data gradient against finite differences and the L L^H = 2 I
identity, and the iteration against the non-expansiveness of a primal-dual step in its
metric (a planted error breaks it), feasibility and objective decrease."""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import prox
from oracle import tv
from problems import make_problem


def test_grad_adjointness_and_norm():
    rng = np.random.default_rng(0)
    U = rng.normal(size=(3, 10, 10))
    G = rng.normal(size=(3, 2, 10, 10))
    assert np.isclose(np.sum(tv.grad(U) * G), np.sum(U * tv.grad_adjoint(G)), rtol=1e-12)
    # Closed forms: the checkerboard is the top eigenvector of grad^T grad with eigenvalue 8;
    # constants are its kernel; a unit ramp in x has d_x = 1 except at the periodic wrap.
    n = 8
    chk = (-1.0) ** np.add.outer(np.arange(n), np.arange(n))
    assert np.allclose(tv.grad_adjoint(tv.grad(chk)), 8.0 * chk)
    assert np.allclose(tv.grad(np.full((n, n), 3.0)), 0.0)
    ramp = np.tile(np.arange(n, dtype=float), (n, 1))
    gx = tv.grad(ramp)[0]
    assert np.allclose(gx[:, :-1], 1.0) and np.allclose(gx[:, -1], -(n - 1))
    # ||grad||^2 = 8 by power iteration from a random start.
    x = rng.normal(size=(n, n))
    for _ in range(300):
        x = tv.grad_adjoint(tv.grad(x))
        x /= np.linalg.norm(x)
    assert np.isclose(np.sum(x * tv.grad_adjoint(tv.grad(x))), 8.0, rtol=1e-6)


def test_group_soft_threshold_is_the_prox_and_moreau():
    from scipy.optimize import minimize
    rng = np.random.default_rng(1)
    G = rng.normal(size=(2, 2, 3, 3))
    t = rng.uniform(0.1, 2.0, size=(2, 3, 3))
    P = tv.group_soft_threshold(G, t)
    for a in range(2):
        for i in range(3):
            for j in range(3):
                x, tt = G[a, :, i, j], t[a, i, j]
                r = minimize(lambda y: 0.5 * np.sum((y - x) ** 2) + tt * np.linalg.norm(y), x * 0.5,
                             method="Nelder-Mead", options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 4000})
                assert np.allclose(P[a, :, i, j], r.x, atol=1e-6)
    # Moreau: x - prox_{t||.||}(x) is the projection of x onto the disc of radius t.
    norm = np.sqrt(np.sum(G * G, axis=1, keepdims=True))
    proj = G * np.minimum(1.0, t[:, None] / norm)
    assert np.allclose(G - P, proj, atol=1e-14)


def test_data_gradient_identities():
    pb = make_problem(8, 60, 1, 1, seed=3)
    uv, w = pb["uv"], pb["w"].astype(np.float64)
    rng = np.random.default_rng(4)
    S = rng.normal(size=(4, 8, 8))
    Y = pb["Y"].astype(np.complex128)
    g = tv.data_gradient(S, uv, w, Y)
    # L L^H = 2 I: the Stokes-domain gradient is half the correlation-domain one.
    half = 0.5 * meas.phi_adjoint(meas.phi(S, uv, w) - Y, uv, w, 8)
    assert np.allclose(g, half, rtol=1e-10, atol=1e-10)
    # Finite differences of 1/2 ||Y L^-1 - Phi S||^2 along a random direction.
    p = tv.TVParams(1.0, 1.0, 1.0, np.zeros(4), np.zeros(4))
    E = rng.normal(size=S.shape)
    h = 1e-5
    fd = (tv.objective(S + h * E, uv, w, Y, p, tv.TV_NC) - tv.objective(S - h * E, uv, w, Y, p, tv.TV_NC)) / (2 * h)
    assert np.isclose(fd, np.sum(g * E), rtol=1e-6)


def _setup(mode, seed=5, mu=(0.02, 0.01, 0.01, 0.005)):
    pb = make_problem(8, 60, 1, 1, seed=seed)
    uv, w, Y = pb["uv"], pb["w"].astype(np.float64), pb["Y"].astype(np.complex128)
    on = meas.op_norm_sq_lanczos(uv, w, 8)
    p = tv.step_sizes(on, mode, mu=list(mu), nu=[0.01, 0.005, 0.005, 0.002])
    rng = np.random.default_rng(seed)
    st = tv.zero_state(8)
    st["S"] = rng.normal(size=(4, 8, 8)) * 0.1
    return uv, w, Y, p, st


@pytest.mark.parametrize("mu", [(0.02, 0.01, 0.01, 0.005), (100.0, 100.0, 100.0, 100.0)])
@pytest.mark.parametrize("mode", [tv.TV, tv.TV_NC, tv.L1TV, tv.L1TV_NC])
def test_iteration_is_nonexpansive_in_its_metric(mode, mu):
    uv, w, Y, p, st = _setup(mode, mu=mu)
    prev = None
    for _ in range(40):
        nxt = tv.tv_iteration(st, uv, w, Y, p, mode)
        d = {k: nxt[k] - st[k] for k in st}
        m = tv.metric_sq(d, p, mode)
        assert m >= -1e-12
        if prev is not None:
            assert m <= prev * (1 + 1e-9) + 1e-18
        prev, st = m, nxt


def test_planted_error_breaks_nonexpansiveness(monkeypatch):
    """A sign error in grad^T (the operator Psi of step 3) must show up (with TV weights
    large enough for the TV dual to matter against the data term)."""
    mode = tv.TV
    uv, w, Y, p, st = _setup(mode, seed=6, mu=(100.0, 100.0, 100.0, 100.0))
    monkeypatch.setattr(tv, "psi", lambda s, m: -tv.grad_adjoint(s["Atv"]))
    ms = []
    for _ in range(100):
        nxt = tv.tv_iteration(st, uv, w, Y, p, mode)
        ms.append(tv.metric_sq({k: nxt[k] - st[k] for k in st}, p, mode))
        st = nxt
    assert any(b > a * (1 + 1e-6) for a, b in zip(ms, ms[1:]))


@pytest.mark.parametrize("mode", [tv.TV, tv.L1TV, tv.TV_NC])
def test_converges_to_a_feasible_lower_objective(mode):
    uv, w, Y, p, st = _setup(mode, seed=7)
    f0 = tv.objective(np.maximum(st["S"], 0), uv, w, Y, p, mode)
    for _ in range(3000):
        st = tv.tv_iteration(st, uv, w, Y, p, mode)
    S = st["S"]
    assert tv.objective(S, uv, w, Y, p, mode) < f0
    if mode in tv.CONSTRAINED:
        # The epigraph split holds the constraint at convergence: a small residual gap here.
        gap = np.sqrt(S[1] ** 2 + S[2] ** 2 + S[3] ** 2) - S[0]
        assert gap.max() <= 2e-3 * np.abs(S).max()
    else:
        assert S[0].min() >= 0.0
    # The TV dual stays in its discs: |A_tv| <= mu per pixel and map (up to the rounding of
    # A~ - rho1 prox(A~ / rho1), whose terms are ~rho1 |grad Xb| >> mu).
    norm = np.sqrt(np.sum(st["Atv"] ** 2, axis=1))
    assert np.all(norm <= p.mu[:, None, None] * (1 + 1e-8))
    if mode in tv.WITH_L1:
        assert np.all(np.abs(st["Al1"]) <= p.nu[:, None, None] * (1 + 1e-8))


def test_step_sizes_meet_the_condition():
    for mode in (tv.TV, tv.TV_NC, tv.L1TV, tv.L1TV_NC):
        p = tv.step_sizes(1e4, mode, mu=[1, 1, 1, 1])
        knorm = p.rho1 * (9.0 if mode in tv.WITH_L1 else 8.0) + (p.rho3 if mode in tv.CONSTRAINED else 0.0)
        assert 1.0 / p.tau - knorm >= 1e4 / 2.0 / 2.0
    assert prox.proj_U_pos(np.array([[-1.0]])).min() == 0.0
