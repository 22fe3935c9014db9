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
    ref_phi = meas.phi(S.astype(np.float64), pb["uv"], pb["w"].astype(np.float64))
    Yr = (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))).astype(np.complex64)
    ref_adj = meas.phi_adjoint(Yr.astype(np.complex128), pb["uv"], pb["w"].astype(np.float64), n)
    with _solver(pb, n, levels) as s:
        for syn, deg, grd in itertools.product(range(2), range(2), range(3)):
            B.ps_set_tuning(s.h, [syn, deg, grd, 0])
            assert B.ps_get_tuning(s.h) == [syn, deg, grd, 0]
            Sg = np.empty((4, n, n), np.float32)
            B.ps_apply_psi(s.h, A, Sg)
            Yg = np.empty((M, 4), np.complex64)
            B.ps_apply_phi(s.h, S, Yg)
            Ag = np.empty((4, n, n), np.float32)
            B.ps_apply_phi_adjoint(s.h, Yr, Ag)
            assert rel_err(Sg, ref_psi) <= 1e-6, (syn, deg, grd)
            assert rel_err(Yg, ref_phi) <= OP_TOL, (syn, deg, grd)
            assert rel_err(Ag, ref_adj) <= OP_TOL, (syn, deg, grd)


def test_set_tuning_rejects_unknown_choices():
    pb = make_problem(32, 500, 2, 1, seed=13)
    with _solver(pb, 32, 2) as s:
        for bad in ([2, 0, 0, 0], [0, -1, 0, 0], [0, 0, 3, 0], [0, 0, 0, 1]):
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
            if slot in ("synthesis", "degrid", "grid"):
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
