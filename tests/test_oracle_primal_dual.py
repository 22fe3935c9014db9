"""Pins of the oracle's Algorithm 1/2 against convergence theory and the constraint set."""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import primal_dual as pd
from oracle import prox
from oracle import wavelets as wav
from paper_1801_02417_gb300 import inputs


def _problem(n=16, M=200, levels=2, nblocks=2, seed=1, snr=30.0, omega=2.0):
    W = inputs.Workload("tiny", n, M, 6, 40, levels, nblocks, 0, 0, snr, 0, seed)
    uv = inputs.uv_coverage(W, omega_max=omega)
    w = inputs.visibility_weights(M, seed, 0.3)
    Strue = inputs.stokes_source(n, seed)
    Yc = meas.phi(Strue, uv, w)
    sig = inputs.sigma_for_snr(Yc, snr)
    Y = Yc + inputs.complex_noise(M, sig, seed)
    off = inputs.block_offsets(M, nblocks)
    eps = np.array([meas.chi2_epsilon(int(off[b + 1] - off[b]), sig) for b in range(nblocks)])
    return pd.Problem(n, levels, uv, w, Y, off, eps), Strue


def _metric_sequence(prob, p, mode, T, iters, st=None, iteration=pd.pd_iteration):
    st = st or pd.zero_state(prob.n, prob.Y.shape[0])
    out = []
    for _ in range(iters):
        st2 = iteration(st, prob, T, p, mode)
        out.append(pd.metric_sq(*(st2[k] - st[k] for k in "SZABCD"), prob, p, mode))
        st = st2
    return np.array(out), st


@pytest.mark.parametrize("mode", [pd.POLARIZED, pd.NO_CONSTRAINT, pd.NNLS, pd.SOC])
def test_fixed_point_residual_non_increasing(mode):
    """Algorithm 1 is a proximal-point step in the metric M, so ||z_{k+1} - z_k||_M never grows."""
    prob, _ = _problem()
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    p = pd.step_sizes(on, mode)
    T = 2e-3 * np.ones((4, 9, prob.n, prob.n))
    ds, _ = _metric_sequence(prob, p, mode, T, 40)
    assert ds[0] > 0
    # Rounding floor: once converged to machine precision the metric is noise.
    assert np.all(np.diff(ds) <= 1e-10 * ds[:-1] + 1e-24 * ds[0]), ds


def test_planted_sign_error_breaks_monotonicity():
    """A wrong sign on C in step 3 must be caught by the metric pin above."""
    prob, _ = _problem()
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    p = pd.step_sizes(on, pd.POLARIZED)
    T = 2e-3 * np.ones((4, 9, prob.n, prob.n))

    def wrong(st, prob, T, p, mode):
        st = dict(st)
        st["C"] = -st["C"]
        out = pd.pd_iteration(st, prob, T, p, mode)
        return out
    rng = np.random.default_rng(0)
    st0 = pd.zero_state(prob.n, prob.Y.shape[0])
    st0["C"] = rng.normal(size=st0["C"].shape)
    ds, _ = _metric_sequence(prob, p, pd.POLARIZED, T, 30, st=st0, iteration=wrong)
    assert np.any(np.diff(ds) > 1e-6 * ds[:-1])


def test_planted_cone_sign_error_breaks_monotonicity_in_soc_mode():
    """A wrong sign on C in step 3 of the direct cone variant is caught by the same metric pin."""
    prob, _ = _problem()
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    p = pd.step_sizes(on, pd.SOC)
    T = 2e-3 * np.ones((4, 9, prob.n, prob.n))

    def wrong(st, prob, T, p, mode):
        st = dict(st)
        st["C"] = -st["C"]
        return pd.pd_iteration(st, prob, T, p, mode)
    rng = np.random.default_rng(1)
    st0 = pd.zero_state(prob.n, prob.Y.shape[0])
    st0["C"] = rng.normal(size=st0["C"].shape)
    ds, _ = _metric_sequence(prob, p, pd.SOC, T, 30, st=st0, iteration=wrong)
    assert np.any(np.diff(ds) > 1e-6 * ds[:-1])


def test_soc_and_epigraph_split_solve_the_same_problem():
    """Both variants minimise sum T |Psi^dagger S| over P and the data balls: at convergence they
    are feasible, reach the same objective and (the minimiser being unique here) the same maps."""
    prob, _ = _problem(n=16, M=300, levels=2, nblocks=1, seed=3)
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    T = 1e-2 * np.ones((4, 9, prob.n, prob.n))
    out = {}
    for mode in (pd.POLARIZED, pd.SOC):
        st = pd.run(pd.zero_state(prob.n, 300), prob, T, pd.step_sizes(on, mode), 1200, mode)
        S = st["S"]
        assert np.all(pd.residual_norms(S, prob) <= 1.005 * prob.eps)
        pv = -S[0] + np.sqrt(np.sum(S[1:] ** 2, axis=0))
        assert pv.max() <= 1e-4 * S[0].max()
        out[mode] = (S, float(np.sum(T * np.abs(wav.psi_adjoint(S, prob.levels)))))
    (Sa, fa), (Sb, fb) = out[pd.POLARIZED], out[pd.SOC]
    assert abs(fa - fb) <= 1e-3 * fa
    assert np.linalg.norm(Sa - Sb) <= 1e-2 * np.linalg.norm(Sa)


def test_polarized_solution_is_feasible_and_fits_data():
    """At convergence: ||phi S - Y||_b <= (1 + theta) eps_b and S in P (Section 5.5 stop rules)."""
    prob, Strue = _problem(n=16, M=300, levels=2, nblocks=1, seed=3)
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    T = 1e-2 * np.ones((4, 9, prob.n, prob.n))
    st = pd.run(pd.zero_state(prob.n, 300), prob, T, pd.step_sizes(on, pd.POLARIZED), 2500)
    res = pd.residual_norms(st["S"], prob)
    assert np.all(res <= 1.005 * prob.eps), (res, prob.eps)
    pv = -st["S"][0] + np.sqrt(np.sum(st["S"][1:] ** 2, axis=0))
    assert pv.max() <= 1e-4 * st["S"][0].max()
    # The dual variables of the epigraph sit on the polar cones at the fixed point.
    assert np.all(st["C"][0] + st["D"][0] <= 1e-9)


def test_gamma_only_rescales_duals():
    """gamma only affects convergence speed (Section 4.2): two gammas reach the same minimum of ||Psi^dag S||_W,1."""
    prob, _ = _problem(n=8, M=120, levels=1, nblocks=1, seed=5)
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    Wt = np.ones((4, 9, 8, 8))
    vals = []
    for gamma in (3e-2, 1e-1):
        st = pd.run(pd.zero_state(8, 120), prob, gamma * Wt, pd.step_sizes(on, pd.POLARIZED), 6000)
        vals.append(float(np.sum(np.abs(wav.psi_adjoint(st["S"], 1)))))
        assert np.all(pd.residual_norms(st["S"], prob) <= 1.01 * prob.eps)
    assert abs(vals[0] - vals[1]) <= 5e-3 * vals[0], vals


def test_soft_threshold_step_keeps_dual_in_box():
    """After step 6, |A| <= gamma W element-wise (clamp identity of the soft-threshold step)."""
    prob, _ = _problem()
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    p = pd.step_sizes(on, pd.POLARIZED)
    rng = np.random.default_rng(9)
    T = np.abs(rng.normal(size=(4, 9, 16, 16))) * 1e-2
    st = pd.run(pd.zero_state(16, 200), prob, T, p, 5)
    assert np.all(np.abs(st["A"]) <= T * (1 + 1e-12))


def test_nnls_mode_keeps_other_variables_zero_and_I_nonnegative():
    prob, _ = _problem()
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    st = pd.run(pd.zero_state(16, 200), prob, np.zeros((4, 9, 16, 16)), pd.step_sizes(on, pd.NNLS), 20, pd.NNLS)
    for k in "ZACD":
        assert not np.any(st[k])
    assert st["S"][0].min() >= 0.0


def test_reweight_formula_bounds():
    rng = np.random.default_rng(4)
    S = rng.normal(size=(4, 16, 16))
    W = pd.reweight(S, 2, 0.5)
    assert W.shape == (4, 9, 16, 16)
    assert np.all((W > 0) & (W <= 1.0))
    c = np.abs(wav.psi_adjoint(S, 2))
    assert np.allclose(W * (0.5 + c), 0.5)


def test_reweight_hand_computed_haar_and_constant_maps():
    """Eq. weights W = delta / (delta + |Psi^dagger S|) on maps whose SARA coefficients are known in
    closed form. A constant map c: every Daubechies basis puts c 2^L (the filters sum to sqrt 2
    per axis) in its coarsest approximation block and zero in every detail, the Dirac basis c
    everywhere; scaled by 1/3. A point of value v at pixel (0, 0) in the Haar basis (db1):
    level-1 details v/2 at (0, n/2), (n/2, 0), (n/2, n/2), level-2 details and approximation
    v/4 at (0, n/4), (n/4, 0), (n/4, n/4), (0, 0); zero elsewhere."""
    n, L, delta = 8, 2, 0.05
    consts = np.array([1.0, -0.5, 0.25, 2.0])
    S = consts[:, None, None] * np.ones((4, n, n))
    W = pd.reweight(S, L, delta)
    for i, c in enumerate(consts):
        assert np.allclose(W[i, 0], delta / (delta + abs(c) / 3.0), rtol=1e-12)
        for b in range(1, 9):
            expect = np.ones((n, n))
            expect[: n >> L, : n >> L] = delta / (delta + abs(c) * 2 ** L / 3.0)
            assert np.allclose(W[i, b], expect, rtol=1e-12, atol=1e-12), (i, b)
    v = 1.5
    S = np.zeros((4, n, n))
    S[:, 0, 0] = v
    W = pd.reweight(S, L, delta)
    mag = np.zeros((n, n))
    for (r, c) in ((0, n // 2), (n // 2, 0), (n // 2, n // 2)):
        mag[r, c] = v / 2
    for (r, c) in ((0, n // 4), (n // 4, 0), (n // 4, n // 4), (0, 0)):
        mag[r, c] = v / 4
    assert np.allclose(W[0, 1], delta / (delta + mag / 3.0), rtol=1e-12)
    dirac = np.zeros((n, n))
    dirac[0, 0] = v
    assert np.allclose(W[0, 0], delta / (delta + dirac / 3.0), rtol=1e-12)


def test_zeta_threshold_against_the_dense_operator():
    """zeta = 3 rms(Stokes I part of phi^dagger(Y - phi S)) / PSF peak, with the adjoint taken as the
    transpose of the dense real matrix of phi and the PSF peak as its (I centre, I centre) Gram
    entry, which the brightness rows of L fix at 2 sum w_m^2 (|L_I,RR|^2 + |L_I,LL|^2 = 2)."""
    prob, Strue = _problem(n=8, M=40, levels=1, nblocks=1, seed=2)
    n, N = 8, 64
    P = meas.phi_dense(prob.uv, prob.w, n)
    c = (n // 2) * n + n // 2
    peak = float(P[:, c] @ P[:, c])
    assert abs(peak - 2.0 * np.sum(prob.w ** 2)) <= 1e-10 * peak
    S = 0.8 * Strue
    r = prob.Y - meas.phi(S, prob.uv, prob.w)
    img = (P.T @ np.concatenate([r.real.ravel(), r.imag.ravel()]))[:N]
    zeta = 3.0 * np.sqrt(np.mean(img ** 2)) / peak
    assert abs(pd.zeta_threshold(S, prob, 3.0) - zeta) <= 1e-10 * zeta


def test_solve_follows_the_algorithm2_schedule(monkeypatch):
    """Algorithm 2 with the NNLS start: iterations // (reweights + 1) per cycle, the first in NNLS
    mode (g = 0, tau = 0.99 / (rho2 ||phi||^2)), then one reweight before each later cycle with
    delta^(1) = 0.1 max |Psi^dagger S_nnls| halved at every reweight (Section 4.3.4)."""
    prob, _ = _problem(n=8, M=60, levels=1, nblocks=1, seed=6)
    on = meas.op_norm_sq(prob.uv, prob.w, prob.n)
    runs, deltas = [], []
    real_run, real_rw = pd.run, pd.reweight

    def spy_run(st, prob_, T, p, iters, mode=pd.POLARIZED):
        runs.append((mode, iters, float(np.max(np.abs(T))), p.tau))
        return real_run(st, prob_, T, p, iters, mode)

    def spy_rw(S, levels, delta):
        deltas.append(delta)
        return real_rw(S, levels, delta)
    monkeypatch.setattr(pd, "run", spy_run)
    monkeypatch.setattr(pd, "reweight", spy_rw)
    gamma = 0.02
    pd.solve(prob, iterations=14, reweights=3, gamma=gamma, opnorm_sq=on)
    assert [r[0] for r in runs] == [pd.NNLS, pd.POLARIZED, pd.POLARIZED, pd.POLARIZED]
    assert [r[1] for r in runs] == [3, 3, 3, 3]
    assert runs[0][2] == 0.0 and abs(runs[0][3] - 0.99) < 1e-12
    assert all(0 < r[2] <= gamma and abs(r[3] - 0.99 / 3.0) < 1e-12 for r in runs[1:])
    S_nnls = real_run(pd.zero_state(8, 60), prob, np.zeros((4, 9, 8, 8)), pd.step_sizes(on, pd.NNLS), 3,
                      pd.NNLS)["S"]
    d1 = 0.1 * float(np.max(np.abs(wav.psi_adjoint(S_nnls, 1))))
    assert np.allclose(deltas, [d1, d1 / 2, d1 / 4], rtol=1e-12)


def test_relative_change_and_stop_rule():
    """Eq. stop_crit per map with a zero map (V in the paper) that stays zero contributing 0 and one
    that leaves zero contributing inf; the three criteria of Section 5.5 on constructed states."""
    rng = np.random.default_rng(3)
    S0 = rng.normal(size=(4, 8, 8))
    S0[3] = 0.0
    S1 = S0 * (1.0 + np.array([1e-3, 2e-3, 3e-3, 0.0]))[:, None, None]
    assert np.allclose(pd.relative_change(S1, S0), [1e-3, 2e-3, 3e-3, 0.0])
    S2 = S1.copy()
    S2[3, 0, 0] = 1e-9
    assert np.isinf(pd.relative_change(S2, S0)[3])
    # Noise-free data of a feasible source: its residual is 0 <= (1 + theta) eps and N_p = 0.
    prob, Strue = _problem(n=16, M=200, levels=2, nblocks=2, seed=8)
    prob = pd.Problem(prob.n, prob.levels, prob.uv, prob.w, meas.phi(Strue, prob.uv, prob.w), prob.offsets,
                      prob.eps)
    st = pd.stop_rule(Strue * (1 + 1e-6), Strue, prob, rel_tol=1e-5)
    assert st["rel"] and st["resid"] and st["np"] and st["converged"] and st["N_p"] == 0.0
    st = pd.stop_rule(Strue * (1 + 1e-4), Strue, prob, rel_tol=1e-5)
    assert not st["rel"] and not st["converged"]
    # Eq. stop_crit as printed (I, Q, U) ignores a change confined to V.
    Sv = Strue.copy()
    Sv[3] *= 1.01
    assert pd.stop_rule(Sv, Strue, prob, rel_tol=1e-5, maps=3)["rel"]
    assert not pd.stop_rule(Sv, Strue, prob, rel_tol=1e-5, maps=4)["rel"]
    # Far from the data: the fit criterion fails.
    assert not pd.stop_rule(0.5 * Strue, 0.5 * Strue, prob)["resid"]
    # Q made larger than I on 2% of the pixels (beyond zeta): N_p = 2 > 0.5 fails with the constraint only.
    bad = Strue.copy()
    idx = np.unravel_index(np.argsort(Strue[0], axis=None)[-5:], (16, 16))
    bad[1][idx] = bad[0][idx] + 10.0
    st = pd.stop_rule(bad, bad, prob)
    assert abs(st["N_p"] - 100.0 * 5 / 256) < 1e-12 and not st["np"]
    assert pd.stop_rule(bad, bad, prob, constrained=False)["np"]


def test_stats_helpers():
    prob, Strue = _problem()
    assert pd.violation_count(Strue, 0.0) == 0
    bad = Strue.copy()
    bad[1, 3, 3] = bad[0, 3, 3] + 1.0
    assert pd.violation_count(bad, 1e-3) == 1
    rc = pd.relative_change(Strue * 1.1, Strue)
    assert np.allclose(rc, 0.1)
