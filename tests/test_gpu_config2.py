"""The 256 x 256 workload (M = 50,000 rows from 10 stations, 8 l2 blocks, 4 levels) on the GPU
against the FP64 oracle.

* Ten iterations of Algorithm 1 from a seeded random state: every array of the state (S, Z, A,
  B, C, D) within 2e-5 per iteration (the per-operator bound composed over the nonexpansive
  steps), computed by the oracle in the test (~5 s per oracle iteration).
* The full Algorithm 2 solve (500 iterations, 5 reweights, NNLS start) against the oracle's
  result stored in tests/golden/img256_m50k_solve.npz by tests/golden/make_img256_solve.py
  (the direct-DFT oracle needs ~45 min for it): each Stokes map within 1e-3 relative l2 and the
  same violation count N_p at the same zeta.
"""
import os

import numpy as np
import pytest

from oracle import primal_dual as opd
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300 import inputs
from paper_1801_02417_gb300.solver import PolarizedSARA, Schedule
from problems import input_checksums, make_problem, rel_err

pytestmark = pytest.mark.gpu

WL = inputs.WORKLOADS["img256_m50k"]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "img256_m50k_solve.npz")


@pytest.fixture(scope="module")
def cfg2():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    pb = make_problem(WL.n, WL.M, WL.levels, WL.nblocks, seed=WL.seed, stations=WL.stations, weight_spread=0.0)
    gold = dict(np.load(GOLDEN))
    for k, v in input_checksums(pb).items():
        assert abs(v - float(gold[k])) <= 1e-9 * abs(float(gold[k])), (k, v, float(gold[k]))
    return pb, gold


def test_ten_iterations_from_random_state_match_oracle(cfg2):
    pb, gold = cfg2
    n, M, L = WL.n, WL.M, WL.levels
    prob = pb["prob"]
    p = opd.step_sizes(float(gold["opnorm_sq"]), opd.POLARIZED)
    st = inputs.random_state(n, M, 41, 0.05)
    st32 = {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32)) for k, v in st.items()}
    W = np.random.default_rng(42).uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.02
    with PolarizedSARA(n, L, tau=p.tau, rho1=p.rho1, rho2=p.rho2, rho3=p.rho3) as s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        assert abs(s.params()["opnorm_sq"] - float(gold["opnorm_sq"])) <= 1e-5 * float(gold["opnorm_sq"])
        s.set_sara_weights(W, gamma)
        s.set_state(st32)
        s.pd_iterate(10)
        got = s.get_state()
    ref = {k: v.astype(np.complex128 if k == "B" else np.float64) for k, v in st32.items()}
    T = gamma * W.astype(np.float64)
    for _ in range(10):
        ref = opd.pd_iteration(ref, prob, T, p, opd.POLARIZED)
    for k in "SZABCD":
        err = rel_err(got[k], ref[k])
        assert err <= 2e-5 * 10, (k, err)


def test_full_solve_matches_stored_oracle_solve(cfg2):
    pb, gold = cfg2
    n, L = WL.n, WL.levels
    with PolarizedSARA(n, L, rho2=float(gold["rho2"])) as s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        S = s.solve(Schedule(int(gold["iterations"]), int(gold["reweights"]), float(gold["gamma"])))
        st = s.stats()
    ref = gold["S"]
    errs = [rel_err(S[i], ref[i]) for i in range(4)]
    assert max(errs) <= 1e-3, errs
    assert st["violations"] == opd.violation_count(ref, st["zeta"])
    assert np.allclose(st["block_residual"], gold["block_residual"], rtol=1e-3)
