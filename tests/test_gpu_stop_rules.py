"""Stopping rules, boundary defaults and failure reporting of the C ABI on the GPU.

The relative change of Eq. stop_crit and the three criteria of Section 5.5 are compared
with the FP64 oracle on the same FP32 states; the chi^2 radii from sigma (Section 5.1)
and the default gamma with the oracle's formulas; a NaN planted in the state comes back
as PS_ENONFINITE; and the bounded in-kernel waits, given a zero poll budget, give up,
report PS_ETIMEOUT and leave the handle usable.
"""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import primal_dual as opd
from oracle import wavelets as wav
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300 import inputs
from paper_1801_02417_gb300.solver import PolarizedSARA
from problems import make_problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    B.lib()


def _handle(pb, n, levels, **kw):
    s = PolarizedSARA(n, levels, **kw)
    s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
    return s


@pytest.mark.parametrize("tols", [dict(), dict(rel_tol=1.0, resid_tol=100.0, np_tol=100.0),
                                  dict(rel_tol=1.0, resid_tol=100.0, np_tol=100.0, stop_maps=3)])
def test_rel_change_and_stop_flags_match_oracle(tols):
    """Eq. stop_crit per map (V included, or I, Q, U as printed) and the PS_STOP_* flags of
    Section 5.5 against the oracle's stop_rule on the same FP32 states: default tolerances
    (nothing but N_p met after 20 iterations from zero) and loose ones (all met, converged)."""
    n, levels = 32, 3
    pb = make_problem(n, 1500, levels, 4, seed=31)
    prob = pb["prob"]
    with _handle(pb, n, levels, **tols) as s:
        s.set_sara_weights(None, 0.0)
        s.pd_iterate(20)
        S_old = s.get_stokes().astype(np.float64)
        st = s.pd_iterate(1, stats=True)
        S_new = s.get_stokes().astype(np.float64)
        rc = B.ps_get_rel_change(s.h)
        cfg = s.config()
    ref_rc = opd.relative_change(S_new, S_old)
    assert np.all(np.isfinite(ref_rc)) and np.all(ref_rc > 0)
    assert np.allclose(st["rel_change"], ref_rc, rtol=1e-5)
    assert np.allclose(rc, ref_rc, rtol=1e-5)
    ref = opd.stop_rule(S_new, S_old, prob, cfg.rel_tol, cfg.resid_tol, cfg.np_tol, cfg.zeta_sigma, True,
                        maps=cfg.stop_maps)
    assert cfg.stop_maps == tols.get("stop_maps", 4)
    flags = {"rel": B.PS_STOP_REL, "resid": B.PS_STOP_RESID, "np": B.PS_STOP_NP}
    for k, bit in flags.items():
        assert bool(st["stop_flags"] & bit) == ref[k], (k, st, ref)
    assert st["converged"] == ref["converged"]
    if not tols:
        assert (cfg.rel_tol, cfg.resid_tol, cfg.np_tol, cfg.zeta_sigma, cfg.stop_maps) == (1e-5, 5e-3, 0.5, 3.0, 4)
        assert not st["converged"]
    else:
        assert st["converged"]


def test_stop_rule_without_constraint_ignores_np():
    """In PS_NO_CONSTRAINT the N_p criterion does not apply (Section 5.5 adds it with the constraint)."""
    n, levels = 32, 2
    pb = make_problem(n, 900, levels, 1, seed=32)
    with _handle(pb, n, levels, mode=B.PS_NO_CONSTRAINT, np_tol=1e-9) as s:
        s.set_sara_weights(None, 0.0)
        # |Q| > I = 0 everywhere, far above zeta (3 rms of the Stokes I residual image in units of
        # the PSF peak, which Q does not enter since L L^H = 2 I): N_p = 100 %.
        bad = np.zeros((4, n, n), np.float32)
        bad[1] = 1e4
        s.set_state({"S": bad})
        st = s.stats()
        assert st["violations"] == n * n
        assert st["stop_flags"] & B.PS_STOP_NP
        s.set_mode(B.PS_POLARIZED)
        assert not (s.stats()["stop_flags"] & B.PS_STOP_NP)


def test_eps_from_noise_sigma_is_the_chi2_bound():
    """eps = NULL: the radii of Section 5.1 from cfg.noise_sigma. The iteration then matches a
    handle given the oracle's chi^2 radii explicitly; without noise_sigma the call is refused."""
    n, levels = 32, 3
    pb = make_problem(n, 1500, levels, 4, seed=33)
    a = PolarizedSARA(n, levels, noise_sigma=pb["sigma"])
    b = _handle(pb, n, levels)
    with a, b:
        a.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], None)
        for s in (a, b):
            s.set_sara_weights(None, 0.0)
            s.pd_iterate(40)
        assert rel_err(a.get_stokes(), b.get_stokes()) <= 1e-5
        sa, sb = a.stats(), b.stats()
        assert sa["stop_flags"] == sb["stop_flags"]
    with PolarizedSARA(n, levels) as c:
        with pytest.raises(B.PolsaraError) as e:
            c.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], None)
        assert e.value.status == B.PS_EINVAL


def test_default_gamma_matches_its_definition():
    """cfg.gamma = 0: gamma = 1e-3 max|Psi^dagger phi^dagger Y| / ||phi||^2, with the oracle's
    phi^dagger, Psi^dagger and Lanczos estimate; the thresholds start at gamma W, W = 1."""
    n, levels = 32, 3
    pb = make_problem(n, 1200, levels, 2, seed=34)
    prob = pb["prob"]
    on = meas.op_norm_sq_lanczos(pb["uv"], prob.w, n)
    ref = 1e-3 * float(np.max(np.abs(wav.psi_adjoint(meas.phi_adjoint(prob.Y, pb["uv"], prob.w, n), levels)))) / on
    with _handle(pb, n, levels) as s:
        g = s.config().gamma
        T = s.get_sara_weights()
    assert abs(g - ref) <= 1e-4 * ref
    assert np.allclose(T, g, rtol=1e-6)
    with _handle(pb, n, levels, gamma=0.125) as s:
        assert s.config().gamma == 0.125
        assert np.allclose(s.get_sara_weights(), 0.125)


@pytest.mark.parametrize("plane", ["S", "C"])
def test_nonfinite_state_is_reported(plane):
    """A NaN planted through ps_set_state (in S, or in the dual C, which reaches S in one iteration)
    is reported as PS_ENONFINITE by the relative-change sums, not returned as numbers."""
    n, levels = 32, 2
    pb = make_problem(n, 900, levels, 1, seed=35)
    with _handle(pb, n, levels) as s:
        s.set_sara_weights(None, 0.0)
        s.pd_iterate(3)
        x = np.zeros((4, n, n), np.float32)
        x[1, 5, 7] = np.nan
        s.set_state({plane: x})
        s.pd_iterate(1)
        with pytest.raises(B.PolsaraError) as e:
            B.ps_get_rel_change(s.h)
        assert e.value.status == B.PS_ENONFINITE
        with pytest.raises(B.PolsaraError) as e:
            s.pd_iterate(1, stats=True)
        assert e.value.status == B.PS_ENONFINITE
        # A finite state makes the handle usable again.
        s.set_state({"S": np.zeros((4, n, n), np.float32), "Z": np.zeros((2, n, n), np.float32),
                     "A": np.zeros((4, 9, n, n), np.float32), "B": np.zeros((900, 4), np.complex64),
                     "C": np.zeros((4, n, n), np.float32), "D": np.zeros((2, n, n), np.float32)})
        # From the zero state the first iteration leaves S at zero (every dual is zero) and the
        # second moves it: the relative change is +inf (a map that left zero), and finite after.
        s.pd_iterate(2)
        assert np.all(np.isposinf(B.ps_get_rel_change(s.h)))
        s.pd_iterate(1)
        assert np.all(np.isfinite(B.ps_get_rel_change(s.h)))


@pytest.mark.parametrize("tuning", [[0, 0, 3, 1], [1, 0, 0, 0], [1, 0, 0, 5]])
def test_bounded_wait_gives_up_then_recovers(tuning):
    """With a zero poll budget every bulk-copy wait gives up at once: the CTAs raise the flag,
    drain their copies with the full budget and return; ps_synchronize reports PS_ETIMEOUT.
    With the budget restored the handle iterates like the oracle again. The tunings cover
    every kernel with such a wait (tiled and persistent analysis, the multi-basis level-1
    analysis with one staging set, both synthesis forms, the tensor-core gridding; at 256^2
    with 3 levels, levels 1-2 are tiled and level 2 of the synthesis takes its own tiled
    kernel)."""
    n, M, levels = 256, 2000, 3
    pb = make_problem(n, M, levels, 2, seed=36)
    prob = pb["prob"]
    on = meas.op_norm_sq_lanczos(pb["uv"], prob.w, n)
    p = opd.step_sizes(on, opd.POLARIZED)
    st = inputs.random_state(n, M, 37, 0.05)
    st32 = {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32)) for k, v in st.items()}
    W = np.random.default_rng(38).uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.02
    with _handle(pb, n, levels, tau=p.tau, rho1=p.rho1, rho2=p.rho2, rho3=p.rho3) as s:
        B.ps_set_tuning(s.h, tuning)
        s.set_sara_weights(W, gamma)
        s.set_state(st32)
        s.synchronize()
        B.ps_debug_set_wait_polls(0)
        try:
            s.pd_iterate(1)
            with pytest.raises(B.PolsaraError) as e:
                s.synchronize()
            assert e.value.status == B.PS_ETIMEOUT
        finally:
            B.ps_debug_set_wait_polls(-1)
        s.synchronize()                       # the flag was cleared by the report
        s.set_state(st32)
        s.pd_iterate(2)
        got = s.get_state()
    ref = {k: v.astype(np.complex128 if k == "B" else np.float64) for k, v in st32.items()}
    T = gamma * W.astype(np.float64)
    for _ in range(2):
        ref = opd.pd_iteration(ref, prob, T, p, opd.POLARIZED)
    for k in "SZABCD":
        assert rel_err(got[k], ref[k]) <= 2e-5 * 2, k


def test_fp32_peak_measurement_is_plausible():
    """ps_fp32_peak (the compute ceiling reported beside the HBM roofline): between 10 and 500
    TFLOP/s on one GPU of this class, for packed FP32x2 and scalar FMA chains."""
    for packed in (True, False):
        v = B.ps_fp32_peak(packed)
        assert 1e13 < v < 5e14, (packed, v)


def test_multi_iteration_graph_matches_single_launches():
    """ps_pd_iterate runs of kGraphIters (8) iterations go out as one launch of a graph holding
    them back to back: 19 iterations in one call (two such launches and three single ones)
    leave the same state as 19 calls of one iteration, to the run-to-run spread of the FP32
    atomics (two runs of 19 single launches differ by about 1e-6 in S, Z, B, C, D and 1.5e-5
    in A, where the soft-threshold of the l1 dual passes the spread on to small entries)."""
    n, levels = 32, 3
    pb = make_problem(n, 1500, levels, 4, seed=39)
    st0 = inputs.random_state(n, 1500, 40, 0.05)
    st32 = {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32)) for k, v in st0.items()}
    a, b = _handle(pb, n, levels), _handle(pb, n, levels)
    with a, b:
        for s in (a, b):
            s.set_sara_weights(None, 0.0)
            s.set_state(st32)
        a.pd_iterate(19)
        for _ in range(19):
            b.pd_iterate(1)
        ga, gb = a.get_state(), b.get_state()
    for k in "SZABCD":
        assert rel_err(ga[k], gb[k]) <= (6e-5 if k == "A" else 1e-5), k


def test_rel_change_request_reads_the_iteration_it_follows():
    """ps_rel_change_request after iteration k, then iteration k + 1, then ps_rel_change_result:
    the relative change of iteration k, as a second handle in the same state reads it with
    ps_get_rel_change right after its iteration k (the two handles differ only in the order of
    the FP32 gridding atomics); after the last iteration the asynchronous and the synchronous
    read agree bit for bit. Without a pending request the result call is PS_ESTATE, and a NaN
    in the state comes back from the result as PS_ENONFINITE."""
    n, levels, M = 32, 3, 900
    pb = make_problem(n, M, levels, 2, seed=50)
    st32 = {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32))
            for k, v in inputs.random_state(n, M, 51, 0.05).items()}
    a, b = _handle(pb, n, levels), _handle(pb, n, levels)
    with a, b:
        for s in (a, b):
            s.set_sara_weights(None, 0.02)
            s.set_state(st32)
        with pytest.raises(B.PolsaraError) as e:
            B.ps_rel_change_result(a.h)
        assert e.value.status == B.PS_ESTATE
        got = []
        a.pd_iterate(1)
        B.ps_rel_change_request(a.h)
        for _ in range(4):
            a.pd_iterate(1)
            got.append(B.ps_rel_change_result(a.h))
            B.ps_rel_change_request(a.h)
        got.append(B.ps_rel_change_result(a.h))
        assert np.array_equal(got[-1], B.ps_get_rel_change(a.h))
        ref = []
        for _ in range(5):
            b.pd_iterate(1)
            ref.append(B.ps_get_rel_change(b.h))
        for k in range(5):
            assert np.all(np.isfinite(got[k])) and np.all(got[k] > 0), k
            assert np.allclose(got[k], ref[k], rtol=1e-4, atol=0.0), (k, got[k], ref[k])
        x = np.zeros((4, n, n), np.float32)
        x[2, 3, 4] = np.nan
        a.set_state({"S": x})
        a.pd_iterate(1)
        B.ps_rel_change_request(a.h)
        with pytest.raises(B.PolsaraError) as e:
            B.ps_rel_change_result(a.h)
        assert e.value.status == B.PS_ENONFINITE
