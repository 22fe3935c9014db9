"""Autotuned launch choices: every candidate computes the same operators (parity
with the FP64 oracle for each choice), and the autotuner leaves the iteration's
state and results unchanged."""
import itertools

import numpy as np
import pytest

from oracle import measurement as meas
from oracle import wavelets as wav
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300.solver import PolarizedSARA
from problems import make_problem, rel_err

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    B.lib()


def _solver(pb, n, levels):
    s = PolarizedSARA(n, levels)
    s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
    return s


@pytest.mark.parametrize("n,M,levels", [(64, 3000, 4), (256, 4000, 5)])
def test_every_launch_choice_matches_oracle(n, M, levels):
    pb = make_problem(n, M, levels, 2, seed=11)
    rng = np.random.default_rng(12)
    S = rng.normal(size=(4, n, n)).astype(np.float32)
    A = rng.normal(size=(4, 9, n, n)).astype(np.float32)
    ref_psi = wav.psi(A.astype(np.float64), levels)
    ref_psia = wav.psi_adjoint(S.astype(np.float64), levels)
    ref_phi = meas.phi(S.astype(np.float64), pb["uv"], pb["w"].astype(np.float64))
    Yr = (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))).astype(np.complex64)
    ref_adj = meas.phi_adjoint(Yr.astype(np.complex128), pb["uv"], pb["w"].astype(np.float64), n)
    with _solver(pb, n, levels) as s:
        for syn, deg, grd, ana in itertools.product(range(3), range(3), range(5), range(6)):
            B.ps_set_tuning(s.h, [syn, deg, grd, ana])
            assert B.ps_get_tuning(s.h) == [syn, deg, grd, ana]
            Sg = np.empty((4, n, n), np.float32)
            B.ps_apply_psi(s.h, A, Sg)
            Yg = np.empty((M, 4), np.complex64)
            B.ps_apply_phi(s.h, S, Yg)
            Ag = np.empty((4, n, n), np.float32)
            B.ps_apply_phi_adjoint(s.h, Yr, Ag)
            Cg = np.empty((4, 9, n, n), np.float32)
            B.ps_apply_psi_adjoint(s.h, S, Cg)
            key = (syn, deg, grd, ana)
            assert rel_err(Sg, ref_psi) <= 1e-6, key
            assert rel_err(Cg, ref_psia) <= 1e-6, key
            assert rel_err(Yg, ref_phi) <= OP_TOL, key
            assert rel_err(Ag, ref_adj) <= OP_TOL, key


def test_set_tuning_rejects_unknown_choices():
    pb = make_problem(32, 500, 2, 1, seed=13)
    with _solver(pb, 32, 2) as s:
        for bad in ([3, 0, 0, 0], [0, 3, 0, 0], [0, 0, 5, 0], [0, 0, 0, 6]):
            with pytest.raises(B.PolsaraError) as e:
                B.ps_set_tuning(s.h, bad)
            assert e.value.status == B.PS_EINVAL
        assert B.ps_get_tuning(s.h) == [0, 0, 0, 0]


def test_autotune_keeps_the_state_and_the_iteration():
    """Two solvers from the same start: one autotuned, one on the default choices.
    The autotuner changes nothing in the state, and the next iterations agree within
    the iteration bound of the parity tests (2e-5 per iteration): the candidates
    differ only in the grouping of FP32 partial sums, which the ball factor
    c_b = rho2 (1 - eps/r) amplifies when the block residual r is near eps."""
    n, M, levels = 128, 6000, 4
    pb = make_problem(n, M, levels, 4, seed=14)
    with _solver(pb, n, levels) as a, _solver(pb, n, levels) as b:
        a.pd_iterate(3)
        b.pd_iterate(3)
        before = np.empty((4, n, n), np.float32)
        B.ps_get_stokes(a.h, before)
        picks = B.ps_autotune(a.h, reps=2)
        for slot, (choice, ms) in picks.items():
            assert choice >= 0
            if slot in ("synthesis", "degrid", "grid", "analysis"):
                assert ms > 0
        after = np.empty((4, n, n), np.float32)
        B.ps_get_stokes(a.h, after)
        assert np.array_equal(before, after)
        a.pd_iterate(5)
        b.pd_iterate(5)
        sa = np.empty((4, n, n), np.float32)
        sb = np.empty((4, n, n), np.float32)
        B.ps_get_stokes(a.h, sa)
        B.ps_get_stokes(b.h, sb)
        assert rel_err(sa, sb) <= 2e-5 * 5


@pytest.mark.parametrize("tuning", [[0, 0, 0, 1], [0, 1, 3, 0], [0, 0, 0, 2], [1, 0, 0, 3], [2, 0, 4, 2],
                                    [1, 0, 3, 4], [0, 2, 1, 0], [1, 2, 3, 5]])
def test_forced_launch_choices_iterate_like_oracle(tuning):
    """Forced launch choices inside the iteration against Algorithm 1 of the FP64 oracle
    from a random state: [0, 0, 0, 1] the persistent analysis form (dual update with
    staged A and gamma W, refilled buffers; level 1 is tiled at this size), [0, 1, 3, 0]
    the chunk-per-warp degridding (residual, block sums) and tensor-core gridding forms,
    [0, 0, 0, 2] and [1, 0, 0, 3] the level-1 analysis with the input tile shared by 8 or 4
    bases (both staging sets in use), [2, 0, 4, 2] the persistent finest synthesis level and the
    tensor-core gridding with in-kernel weights, [1, 0, 3, 4] the 512-thread multi-basis analysis,
    [0, 2, 1, 0] the register-capped degridding beside the per-tap gridding, [1, 2, 3, 5] the
    multi-basis analysis with one staging set refilled between bases."""
    from oracle import primal_dual as opd
    from paper_1801_02417_gb300 import inputs
    n, M, levels = 128, 1500, 3
    pb = make_problem(n, M, levels, 2, seed=16)
    prob = pb["prob"]
    on = meas.op_norm_sq_lanczos(pb["uv"], prob.w, n)
    p = opd.step_sizes(on, opd.POLARIZED)
    st = inputs.random_state(n, M, 23, 0.05)
    st32 = {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32)) for k, v in st.items()}
    ref = {k: v.astype(np.complex128 if k == "B" else np.float64) for k, v in st32.items()}
    W = np.random.default_rng(7).uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.02
    T = gamma * W.astype(np.float64)
    s = PolarizedSARA(n, levels, tau=p.tau, rho1=p.rho1, rho2=p.rho2, rho3=p.rho3)
    with s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        s.set_sara_weights(W, gamma)
        B.ps_set_tuning(s.h, tuning)
        s.set_state(st32)
        s.pd_iterate(3)
        for _ in range(3):
            ref = opd.pd_iteration(ref, prob, T, p, opd.POLARIZED)
        got = s.get_state()
    for k in ("S", "Z", "A", "B", "C", "D"):
        assert rel_err(got[k], ref[k]) <= 2e-5 * 3, k


# Relative error of the windowed NUFFT against the exact DFT of the oracle: the ES
# kernel's aliasing error at oversampling 2 falls like exp(-pi W sqrt(1 - 1/2)),
# about 1.5e-5 at W = 5 and below FP32 rounding at W = 9; the bound takes ten times
# that, and never less than the FP32 operator tolerance.
WIDTH_TOL = {5: 1.5e-4, 9: OP_TOL}


@pytest.mark.parametrize("width", [5, 9])
def test_other_kernel_widths_every_choice_match_oracle(width):
    """Kernel widths 5 and 9 (W = 9 runs the CUDA-core gridding forms only; choices 2
    to 4 fall back to 0) on every gridding and degridding launch choice."""
    n, M, levels = 64, 3000, 3
    pb = make_problem(n, M, levels, 2, seed=21)
    rng = np.random.default_rng(22)
    S = rng.normal(size=(4, n, n)).astype(np.float32)
    ref_phi = meas.phi(S.astype(np.float64), pb["uv"], pb["w"].astype(np.float64))
    Yr = (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))).astype(np.complex64)
    ref_adj = meas.phi_adjoint(Yr.astype(np.complex128), pb["uv"], pb["w"].astype(np.float64), n)
    s = PolarizedSARA(n, levels, kernel_width=width)
    with s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        for deg, grd in itertools.product(range(3), range(5)):
            B.ps_set_tuning(s.h, [0, deg, grd, 0])
            Yg = np.empty((M, 4), np.complex64)
            B.ps_apply_phi(s.h, S, Yg)
            Ag = np.empty((4, n, n), np.float32)
            B.ps_apply_phi_adjoint(s.h, Yr, Ag)
            assert rel_err(Yg, ref_phi) <= WIDTH_TOL[width], (width, deg, grd, rel_err(Yg, ref_phi))
            assert rel_err(Ag, ref_adj) <= WIDTH_TOL[width], (width, deg, grd, rel_err(Ag, ref_adj))
