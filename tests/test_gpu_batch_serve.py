"""Batched iterations and the continuous-batching server give the same results as solo runs.

Kernels of different problems overlap on the device, and gridding adds with
float atomics, so results agree within FP32 rounding, not bit for bit. Batched
iterations are compared at 1e-4 relative l2 per Stokes map. Served requests run
whole reweighting schedules, where the reweighting step (delta from
max |Psi^dagger S|, weights delta / (delta + |Psi^dagger S|)) carries rounding
differences into the thresholds; they are compared at the final-map tolerance,
1e-3 relative l2 per Stokes map (observed differences are ~1e-4, largest on the
faint V map).
"""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import primal_dual as opd
from oracle import wavelets as wav
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300.serve import Policy, Problem, Server, synthesize_problem
from paper_1801_02417_gb300.solver import PolarizedSARA, Schedule, solve_batched
from problems import make_channel_problem, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
TOL_FINAL = 1e-3


@pytest.fixture(scope="module")
def problems():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    specs = [(64, 3, 3000, 1, 1), (128, 4, 12000, 2, 2), (64, 2, 800, 3, 1), (128, 3, 20000, 4, 4)]
    return [synthesize_problem(n, L, M, seed, nb) for (n, L, M, seed, nb) in specs]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _start(p, mode=B.PS_POLARIZED):
    s = PolarizedSARA(p.n, p.levels, mode=mode)
    s.set_measurements(p.uv, p.vis, p.weights, p.offsets, p.eps)
    s.set_sara_weights(None, p.gamma)
    return s


def test_batch_graph_matches_individual_iterations(problems):
    solo = []
    for p in problems:
        with _start(p) as s:
            s.pd_iterate(60)
            solo.append(s.get_stokes())
    ss = [_start(p) for p in problems]
    b = B.ps_batch_create([s.h for s in ss])
    try:
        B.ps_batch_iterate(b, 40)
        B.ps_batch_synchronize(b)
        ss[1].set_mode(B.PS_POLARIZED)          # a state/mode change rebuilds the batch graph
        B.ps_batch_iterate(b, 20)
        B.ps_batch_synchronize(b)
        for s, ref in zip(ss, solo):
            assert _rel(s.get_stokes(), ref) <= TOL
    finally:
        B.ps_batch_destroy(b)
        for s in ss:
            s.close()


@pytest.fixture(scope="module")
def class_problems():
    """Two size classes of several problems each (the batch keeps each class's state in shared
    slabs and runs its per-pixel sweep and SARA transforms as class-wide launches), plus a
    single problem of a third class."""
    specs = [(64, 3, 2500, 11, 1), (64, 3, 4000, 12, 2), (64, 3, 1800, 13, 1), (128, 3, 9000, 14, 2),
             (128, 3, 15000, 15, 4), (32, 2, 900, 16, 1)]
    return [synthesize_problem(n, L, M, seed, nb) for (n, L, M, seed, nb) in specs]


def test_class_fused_batch_matches_individual_iterations(class_problems):
    """Iterations of a batch whose size classes run as class-wide launches (and after the batch
    is destroyed, each handle's own arrays again) against the same iterations one handle at a
    time; a handle switched to another mode takes its class out of the fused launches (still
    correct)."""
    probs = class_problems
    solo = []
    for i, p in enumerate(probs):
        with _start(p) as s:
            s.pd_iterate(30)
            if i == 1:
                s.set_mode(B.PS_SOC)
            s.pd_iterate(20)
            s.set_mode(B.PS_POLARIZED)
            s.pd_iterate(10)
            solo.append(s.get_stokes())
    ss = [_start(p) for p in probs]
    b = B.ps_batch_create([s.h for s in ss])
    try:
        B.ps_batch_iterate(b, 30)
        ss[1].set_mode(B.PS_SOC)              # class (64, 3) no longer uniform: per-handle iterations
        B.ps_batch_iterate(b, 20)
        ss[1].set_mode(B.PS_POLARIZED)        # uniform again: class-wide launches
        B.ps_batch_iterate(b, 10)
        B.ps_batch_synchronize(b)
        for s, ref in zip(ss, solo):
            assert _rel(s.get_stokes(), ref) <= TOL
        dev = [B.ps_device_bytes(s.h) for s in ss]
    finally:
        B.ps_batch_destroy(b)
    try:
        # Back in arrays of their own (the slab bytes return to the handles), still iterating.
        for s, d in zip(ss, dev):
            assert B.ps_device_bytes(s.h) >= d
            s.pd_iterate(2)
            assert np.all(np.isfinite(s.get_stokes()))
    finally:
        for s in ss:
            s.close()


def test_batched_algorithm2_matches_solo_solves(class_problems):
    """Whole Algorithm 2 solves run in lockstep through one batch graph per iteration
    (solver.solve_batched: reweights queued on each handle's stream between batch launches,
    size classes in class-wide launches) give each problem the maps of its solo solve."""
    problems = class_problems
    sch = [Schedule(150, 2, p.gamma) for p in problems]
    solo = []
    for p, sc in zip(problems, sch):
        with _start(p) as s:
            solo.append(s.solve(sc))
    ss = [_start(p) for p in problems]
    try:
        got = solve_batched(ss, sch)
    finally:
        for s in ss:
            s.close()
    for g, r in zip(got, solo):
        for k in range(4):
            assert _rel(g[k], r[k]) <= TOL_FINAL, k


def test_each_request_same_alone_and_in_the_mix(problems):
    pol = Policy(rule="rel", rel_tol=0.0, max_iter=300, reweights=2, check_every=25)   # fixed iteration counts
    alone = {}
    for i, p in enumerate(problems):
        res = Server(hbm_budget=1 << 40, max_active=1, policy=pol).run([(0.0, p)])
        alone[i] = res[0].S
    # All requests together, arriving at once, under a budget that admits them in waves.
    budget = sum(p.footprint() for p in problems[:2])
    res = Server(hbm_budget=budget, max_active=8, policy=pol).run([(0.0, p) for p in problems])
    assert sorted(r.rid for r in res) == list(range(len(problems)))
    for r in res:
        assert r.iterations == 300
        for k in range(4):
            assert _rel(r.S[k], alone[r.rid][k]) <= TOL_FINAL, (r.rid, k)


def test_concurrent_preparation_matches_sequential(problems):
    """The server prepares admitted problems on worker threads: handles created and given
    their measurements concurrently must get the same operator norm and the same phi as
    when prepared one at a time (host-side set-up shares no unsynchronised state)."""
    import concurrent.futures

    def prep(p):
        s = PolarizedSARA(p.n, p.levels)
        s.set_measurements(p.uv, p.vis, p.weights, p.offsets, p.eps)
        return s

    ref = []
    for p in problems:
        with prep(p) as s:
            Y = np.empty((p.uv.shape[0], 4), np.complex64)
            B.ps_apply_phi(s.h, np.ones((4, p.n, p.n), np.float32), Y)
            ref.append((B.ps_get_params(s.h)["opnorm_sq"], Y))
    for _ in range(3):
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(problems)) as ex:
            handles = list(ex.map(prep, problems))
        try:
            for p, s, (on, Yr) in zip(problems, handles, ref):
                Y = np.empty((p.uv.shape[0], 4), np.complex64)
                B.ps_apply_phi(s.h, np.ones((4, p.n, p.n), np.float32), Y)
                # phi (interpolation, no atomics) is deterministic; ||phi||^2 comes from power
                # iterations whose gridding adds with float atomics.
                assert np.array_equal(Y, Yr)
                assert abs(B.ps_get_params(s.h)["opnorm_sq"] - on) <= 1e-5 * on   # stop rule 1e-7, atomics
        finally:
            for s in handles:
                s.close()


def test_live_submissions_resolve_like_solo_runs(problems):
    """Server.start/submit/stop: requests submitted from several threads while the
    scheduler runs resolve their futures with the same maps as solo runs; a request whose
    measurements the library rejects (eps <= 0) fails its own future only."""
    import concurrent.futures
    import dataclasses

    pol = Policy(rule="rel", rel_tol=0.0, max_iter=200, reweights=1, check_every=25)
    alone = [Server(hbm_budget=1 << 40, max_active=1, policy=pol).run([(0.0, p)])[0].S for p in problems]
    bad = dataclasses.replace(problems[0], eps=-np.abs(problems[0].eps))
    budget = sum(p.footprint() for p in problems[:3])
    with Server(hbm_budget=budget, max_active=8, policy=pol) as srv:
        with concurrent.futures.ThreadPoolExecutor(4) as ex:
            futs = list(ex.map(srv.submit, problems + [bad] + problems[::-1]))
        got = [f.result(timeout=300) for f in futs[:len(problems)]]
        with pytest.raises(B.PolsaraError) as e:
            futs[len(problems)].result(timeout=300)
        assert e.value.status == B.PS_EINVAL
        got_rev = [f.result(timeout=300) for f in futs[len(problems) + 1:]]
    with pytest.raises(RuntimeError):
        srv.submit(problems[0])
    assert len({r.rid for r in got + got_rev}) == 2 * len(problems)
    for r, ref in zip(got + got_rev, alone + alone[::-1]):
        assert r.iterations == 200
        for k in range(4):
            assert _rel(r.S[k], ref[k]) <= TOL_FINAL, (r.rid, k)


def test_multifrequency_channels_solved_together_like_alone():
    """A multi-frequency observation as independent per-channel solves (the constraint acts
    at each wavelength on its own): all channels submitted at once to the server give each
    channel the maps of its solo solve, every channel's maps are finite, and the channels'
    visibilities differ as their uv scaling and source spectrum say (not copies)."""
    from paper_1801_02417_gb300.serve import synthesize_channels
    chans = synthesize_channels(64, 3, 2500, 4, seed=31)
    assert not np.allclose(chans[0].vis, chans[-1].vis)
    assert np.allclose(chans[-1].uv, chans[0].uv * (1.1 / 0.9))
    pol = Policy(rule="rel", rel_tol=0.0, max_iter=200, reweights=1, check_every=25)
    alone = [Server(hbm_budget=1 << 40, max_active=1, policy=pol).run([(0.0, p)])[0].S for p in chans]
    res = Server(hbm_budget=1 << 40, max_active=8, policy=pol).run([(0.0, p) for p in chans])
    assert sorted(r.rid for r in res) == list(range(len(chans)))
    for r in res:
        assert np.all(np.isfinite(r.S))
        for k in range(4):
            assert _rel(r.S[k], alone[r.rid][k]) <= TOL_FINAL, (r.rid, k)


def test_multifrequency_channel_solve_matches_oracle():
    """One channel of a multi-frequency observation (scaled uv tracks, power-law spectrum,
    Faraday-rotated Q and U; clean visibilities from the oracle's phi) solved through the server
    on the fixed schedule of the 64 x 64 workload (300 iterations, 3 reweights, NNLS start)
    against the FP64 oracle's Algorithm 2: each Stokes map within 1e-3 relative l2."""
    n, M, L = 64, 2000, 4
    pb = make_channel_problem(n, M, L, nchan=8, chan=6, seed=43)
    prob = pb["prob"]
    on = meas.op_norm_sq_lanczos(pb["uv"], prob.w, n)
    gamma = 1e-3 * float(np.max(np.abs(wav.psi_adjoint(meas.phi_adjoint(prob.Y, pb["uv"], prob.w, n), L)))) / on
    ref = opd.solve(prob, 300, 3, gamma, on)["S"]
    req = Problem(n, L, pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"], gamma)
    pol = Policy(rule="rel", rel_tol=0.0, max_iter=300, reweights=3, check_every=25)
    res = Server(hbm_budget=1 << 40, max_active=4, policy=pol).run([(0.0, req)])
    assert res[0].iterations == 300
    errs = [rel_err(res[0].S[k], ref[k]) for k in range(4)]
    assert max(errs) <= 1e-3, errs


def test_nonfinite_request_fails_alone():
    """A request whose visibilities hold a NaN reaches a non-finite state, which the library's
    FP64 sums report as PS_ENONFINITE: that request's future fails and the others resolve."""
    import dataclasses
    base = synthesize_problem(64, 3, 1500, 44, 1)
    vis = base.vis.copy()
    vis[17, 2] = np.nan
    bad = dataclasses.replace(base, vis=vis)
    pol = Policy(max_iter=200, reweights=1, check_every=20)
    with Server(hbm_budget=1 << 40, max_active=4, policy=pol) as srv:
        futs = [srv.submit(p) for p in (base, bad, base)]
        ok = [futs[0].result(timeout=300), futs[2].result(timeout=300)]
        with pytest.raises(B.PolsaraError) as e:
            futs[1].result(timeout=300)
    assert e.value.status == B.PS_ENONFINITE
    for r in ok:
        assert np.all(np.isfinite(r.S))
