"""Continuous-batching solve server for Polarized SARA requests.

Requests (independent imaging problems) arrive over time. The server admits
them in arrival order while their estimated device footprint
(`ps_estimate_bytes`) fits the memory budget and a slot is free, prepares each
admitted problem on a worker thread (handle creation, row sorting, operator
norm), and keeps every active problem's primal/dual state resident on the
GPU. Each scheduler tick launches `check_every` iterations of every active
problem on its own CUDA stream, so the kernels of different problems overlap on
the device, then evaluates each problem's stopping rule (Section 5.5: the
relative change of Eq. stop_crit, the data fit within (1 + vartheta) eps_b and,
with the constraint, N_p <= varrho) and advances its Algorithm 2 phase: an NNLS
cycle, then up to `reweights` reweighted cycles of Algorithm 1. A request whose
state turns non-finite (PS_ENONFINITE from the library's FP64 sums) fails alone. Finished problems return their
Stokes maps and free their memory, which admits the next requests.

Two front ends share the scheduler: `Server.run(requests)` replays a recorded
arrival schedule, and `Server.start()` / `submit(problem) -> Future` / `stop()`
(or `with Server(...) as srv:`) serves live submissions from any thread.

All arithmetic runs in libpolsara.so; this module only schedules C ABI calls.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import statistics
import threading
import time

import numpy as np

from . import binding as B
from .solver import PolarizedSARA


@dataclasses.dataclass
class Problem:
    n: int
    levels: int
    uv: np.ndarray             # (M, 2) float64, rad/pixel
    vis: np.ndarray            # (M, 4) complex64
    weights: np.ndarray | None
    offsets: np.ndarray        # (nblocks + 1,)
    eps: np.ndarray            # (nblocks,)
    gamma: float

    def footprint(self) -> int:
        return B.ps_estimate_bytes(self.n, self.levels, self.uv.shape[0])


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    iterations: int
    S: np.ndarray

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclasses.dataclass
class Policy:
    rel_tol: float = 1e-4          # Eq. stop_crit tolerance per cycle
    rule: str = "paper"            # "paper": every criterion of Section 5.5; "rel": the relative change only
    maps: int = 4                  # maps of Eq. stop_crit: 3 = I, Q, U as printed, 4 = V included
    max_iter: int = 2000           # per request
    reweights: int = 5             # reweighted cycles after the NNLS cycle
    check_every: int = 20          # iterations between stop-rule checks
    delta_factor: float = 0.1      # delta^(1) = factor * max |Psi^dagger S_nnls|
    delta_decay: float = 0.5


class _Active:
    def __init__(self, rid, prob: Problem, solver: PolarizedSARA, arrival: float, admitted: float, policy: Policy):
        self.rid, self.prob, self.s = rid, prob, solver
        self.arrival, self.admitted = arrival, admitted
        self.policy = policy
        self.cycle = 0               # 0 = NNLS, 1..reweights = reweighted cycles
        self.in_cycle = 0
        self.used = 0
        self.delta = None
        self.per_cycle = max(policy.check_every, policy.max_iter // (policy.reweights + 1))

    def launch(self) -> int:
        k = min(self.policy.check_every, self.per_cycle - self.in_cycle, self.policy.max_iter - self.used)
        if k > 0:
            self.s.pd_iterate(k)
            self.in_cycle += k
            self.used += k
        return k

    def advance(self) -> bool:
        """Check the stop rule after the launched iterations; True when the request is done."""
        if self.policy.rule == "paper":
            met = B.ps_compute_stats(self.s.h, 0.0, self.s.nblocks)["converged"]
        else:
            met = float(np.max(B.ps_get_rel_change(self.s.h)[:self.policy.maps])) <= self.policy.rel_tol
        cycle_done = met or self.in_cycle >= self.per_cycle
        if self.used >= self.policy.max_iter:
            return True
        if not cycle_done:
            return False
        if self.cycle >= self.policy.reweights:
            return True
        if self.cycle == 0:
            self.delta = self.policy.delta_factor * B.ps_max_abs_analysis(self.s.h)
            self.s.set_sara_weights(None, self.prob.gamma)
            self.s.set_mode(B.PS_POLARIZED)
        else:
            self.delta *= self.policy.delta_decay
        self.s.reweight(self.delta)
        self.cycle += 1
        self.in_cycle = 0
        return False


def tuning_key(n: int, M: int) -> tuple:
    """Problems of one image size and the same power-of-two bracket of visibility count share launch choices."""
    return (int(n), int(max(M, 1)).bit_length())


def apply_tuning(s: PolarizedSARA, n: int, M: int, cache: dict, lock: threading.Lock | None = None) -> None:
    """Set the handle's launch choices from the cache, autotuning (ps_autotune) the first of its class."""
    key = tuning_key(n, M)
    if lock is not None:
        lock.acquire()
    try:
        choices = cache.get(key)
        if choices is None:
            B.ps_autotune(s.h, reps=2)
            cache[key] = B.ps_get_tuning(s.h)
        else:
            B.ps_set_tuning(s.h, choices)
    finally:
        if lock is not None:
            lock.release()


class Server:
    """Admission by device footprint, resident state, and overlapping per-problem streams."""

    def __init__(self, hbm_budget: int, max_active: int = 64, policy: Policy | None = None, prep_workers: int = 2,
                 autotune: bool = True):
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.policy = policy or Policy()
        self.prep_workers = prep_workers
        self.autotune = autotune
        self._tuning: dict = {}
        self._tuning_lock = threading.Lock()
        self._thread: threading.Thread | None = None
        self._id_lock = threading.Lock()

    def _prepare(self, prob: Problem) -> PolarizedSARA:
        s = PolarizedSARA(prob.n, prob.levels, mode=B.PS_NNLS, rel_tol=self.policy.rel_tol, stop_maps=self.policy.maps)
        try:
            s.set_measurements(prob.uv, prob.vis, prob.weights, prob.offsets, prob.eps)
            if self.autotune:
                apply_tuning(s, prob.n, prob.uv.shape[0], self._tuning, self._tuning_lock)
        except BaseException:
            s.close()
            raise
        return s

    def run(self, requests: list[tuple[float, Problem]]) -> list[Result]:
        """Serve requests given as (arrival offset in seconds, problem), in real time."""
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        results: list[Result] = []

        def poll(now):
            out = []
            while order and requests[order[0]][0] <= now:
                rid = order.pop(0)
                out.append((rid, requests[rid][0], requests[rid][1]))
            return out

        def next_arrival():
            return requests[order[0]][0] if order else None

        def fail(rid, exc):
            raise exc

        self._schedule(poll, next_arrival, lambda: not order, results.append, fail)
        return results

    # ---- live serving: submit() from any thread while the scheduler runs.
    def __enter__(self) -> "Server":
        self.start()
        return self

    def __exit__(self, *exc) -> None:
        self.stop()

    def start(self) -> None:
        """Start the scheduler on a background thread; requests then come from submit()."""
        import queue
        self._queue = queue.Queue()
        self._closing = threading.Event()
        self._futures: dict = {}
        self._next_id = 0
        self._t0 = time.perf_counter()
        self._thread = threading.Thread(target=self._live_loop, daemon=True)
        self._thread.start()

    def submit(self, prob: Problem) -> concurrent.futures.Future:
        """Queue one solve; the future resolves to its Result (or raises its error)."""
        if self._thread is None or self._closing.is_set():
            raise RuntimeError("server not running: submit() before start() or after stop()")
        fut: concurrent.futures.Future = concurrent.futures.Future()
        with self._id_lock:
            rid = self._next_id
            self._next_id += 1
        self._futures[rid] = fut
        self._queue.put((rid, time.perf_counter() - self._t0, prob))
        return fut

    def stop(self) -> None:
        """Finish every submitted request, then end the scheduler thread."""
        if self._thread is None:
            return
        self._closing.set()
        self._thread.join()
        self._thread = None

    def _live_loop(self) -> None:
        import queue
        waiting: list = []

        def poll(now):
            while True:
                try:
                    waiting.append(self._queue.get_nowait())
                except queue.Empty:
                    break
            out, waiting[:] = list(waiting), []
            return out

        def deliver(r: Result) -> None:
            self._futures.pop(r.rid).set_result(r)

        def fail(rid, exc) -> None:
            self._futures.pop(rid).set_exception(exc)

        def done() -> bool:
            return self._closing.is_set() and self._queue.empty()

        try:
            self._schedule(poll, lambda: None, done, deliver, fail, t0=self._t0)
        except BaseException as e:   # fail every request still waiting
            for f in list(self._futures.values()):
                if not f.done():
                    f.set_exception(e)
            raise

    def _schedule(self, poll, next_arrival, exhausted, deliver, fail, t0: float | None = None) -> None:
        """Admission in arrival order by footprint and free slots, preparation on worker
        threads, ticks of `check_every` iterations of every active problem (each on its own
        stream), stopping rules, delivery. poll(now) returns newly arrived (rid, arrival,
        problem); exhausted() tells that no more will arrive; fail(rid, exc) reports a
        request whose preparation or iterations raised (its memory is released first)."""
        t0 = time.perf_counter() if t0 is None else t0
        pending: list = []
        in_use = 0
        preparing: dict = {}
        active: list[_Active] = []
        with concurrent.futures.ThreadPoolExecutor(self.prep_workers) as pool:
            while True:
                now = time.perf_counter() - t0
                pending.extend(poll(now))
                if not (pending or preparing or active) and exhausted():
                    break
                # Admission in arrival order: footprint within budget and a free slot.
                while pending:
                    rid, arrival, prob = pending[0]
                    fp = prob.footprint()
                    if len(active) + len(preparing) >= self.max_active or (in_use + fp > self.budget and in_use > 0):
                        break
                    pending.pop(0)
                    in_use += fp
                    preparing[pool.submit(self._prepare, prob)] = (rid, arrival, prob, fp, now)
                for fut in [f for f in preparing if f.done()]:
                    rid, arrival, prob, fp, adm = preparing.pop(fut)
                    if fut.exception() is not None:
                        in_use -= fp
                        fail(rid, fut.exception())
                        continue
                    active.append(_Active(rid, prob, fut.result(), arrival, adm, self.policy))
                if not active:
                    if preparing:
                        concurrent.futures.wait(list(preparing), timeout=0.05,
                                                return_when=concurrent.futures.FIRST_COMPLETED)
                    else:
                        nxt = next_arrival()
                        wait = 0.005 if nxt is None else max(0.0, nxt - (time.perf_counter() - t0))
                        time.sleep(min(0.05, wait))
                    continue
                # One tick: launch every active problem (each on its own stream), then check them.
                errors: dict = {}
                for a in active:
                    try:
                        a.launch()
                    except B.PolsaraError as e:
                        errors[a.rid] = e
                still = []
                for a in active:
                    try:
                        if a.rid in errors:
                            raise errors[a.rid]
                        if not a.advance():
                            still.append(a)
                            continue
                        S = a.s.get_stokes()
                    except B.PolsaraError as e:
                        a.s.close()
                        in_use -= a.prob.footprint()
                        fail(a.rid, e)
                        continue
                    a.s.close()
                    in_use -= a.prob.footprint()
                    deliver(Result(a.rid, a.arrival, a.admitted, time.perf_counter() - t0, a.used, S))
                active = still


def summarize(results: list[Result]) -> dict:
    if not results:
        return {"solves": 0}
    lat = sorted(r.latency for r in results)
    span = max(r.finished for r in results) - min(r.arrival for r in results)

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
    return {"solves": len(results), "solves_per_s": len(results) / span if span > 0 else None,
            "p50_s": pct(50), "p99_s": pct(99), "mean_s": statistics.mean(lat),
            "iterations_mean": statistics.mean(r.iterations for r in results)}


def chi2_epsilon(M_b: int, sigma: float) -> float:
    """l2-ball radius of Section 5.1: eps^2 = (8M + 2 sqrt(16M)) sigma^2 / 2."""
    dof = 8.0 * M_b
    return float(np.sqrt((dof + 2.0 * np.sqrt(2.0 * dof)) * sigma * sigma / 2.0))


def synthesize_problem(n: int, levels: int, M: int, seed: int, nblocks: int = 1, snr_db: float = 30.0,
                       n_compact: int = 0, gamma_factor: float = 1e-3) -> Problem:
    """A seeded request whose clean visibilities come from the library's own phi.

    uv tracks and the source come from `inputs`; the noise matches `snr_db`; the
    l2 radii are the chi^2 bounds; gamma = gamma_factor * max |Psi^dagger phi^dagger Y| / ||phi||^2
    (image units: phi^dagger phi peaks at ||phi||^2; gamma does not change the minimiser).
    """
    from . import inputs
    stations = 8
    pairs = stations * (stations - 1) // 2
    while pairs * 16 < M:
        stations += 2
        pairs = stations * (stations - 1) // 2
    wl = inputs.Workload("request", n, M, stations, M // pairs + 2, levels, nblocks, 0, 0, snr_db, n_compact, seed)
    uv = inputs.uv_coverage(wl)
    w = np.ones(M, np.float32)
    truth = inputs.stokes_source(n, seed, n_compact).astype(np.float32)
    off = inputs.block_offsets(M, nblocks)
    with PolarizedSARA(n, levels) as s:
        s.set_measurements(uv, np.zeros((M, 4), np.complex64), w, off, np.ones(nblocks))
        clean = np.empty((M, 4), np.complex64)
        B.ps_apply_phi(s.h, truth, clean)
        sigma = inputs.sigma_for_snr(clean, snr_db)
        Y = (clean + inputs.complex_noise(M, sigma, seed)).astype(np.complex64)
        B.ps_set_visibilities(s.h, Y)
        dirty = np.empty((4, n, n), np.float32)
        B.ps_apply_phi_adjoint(s.h, Y, dirty)
        s.set_state({"S": dirty})
        gamma = gamma_factor * B.ps_max_abs_analysis(s.h) / B.ps_get_params(s.h)["opnorm_sq"]
    eps = np.array([chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(nblocks)])
    return Problem(n, levels, uv, Y, w, off, eps, gamma)


def synthesize_channels(n: int, levels: int, M: int, nchan: int, seed: int, nblocks: int = 1,
                        frac_bw: float = 0.2, alpha: float = -0.7, rm_peak: float = 2.0, snr_db: float = 30.0,
                        gamma_factor: float = 1e-3) -> list[Problem]:
    """Multi-frequency (hyperspectral) observation of one polarized source as independent
    per-channel problems (the polarization constraint acts at each wavelength on its own).

    One uv track set at the reference frequency, scaled per channel; the source follows a
    power law of index `alpha` with Faraday rotation by a smooth RM lambda_0^2 map of peak
    `rm_peak` rad; clean visibilities from the library's phi, noise at `snr_db` per channel,
    chi^2 radii and gamma per channel as in `synthesize_problem`.
    """
    from . import inputs
    stations = 8
    pairs = stations * (stations - 1) // 2
    while pairs * 16 < M:
        stations += 2
        pairs = stations * (stations - 1) // 2
    wl = inputs.Workload("channels", n, M, stations, M // pairs + 2, levels, nblocks, 0, 0, snr_db, 0, seed)
    ratios = inputs.channel_ratios(nchan, frac_bw)
    uv0 = inputs.uv_coverage(wl, omega_max=inputs.EHT_OMEGA_MAX / float(ratios.max()))
    S0 = inputs.stokes_source(n, seed)
    rm = inputs.rotation_measure_map(n, seed, rm_peak)
    w = np.ones(M, np.float32)
    off = inputs.block_offsets(M, nblocks)
    out = []
    for c, ratio in enumerate(ratios):
        uv = inputs.channel_uv(uv0, float(ratio))
        truth = inputs.channel_stokes(S0, float(ratio), alpha, rm).astype(np.float32)
        with PolarizedSARA(n, levels) as s:
            s.set_measurements(uv, np.zeros((M, 4), np.complex64), w, off, np.ones(nblocks))
            clean = np.empty((M, 4), np.complex64)
            B.ps_apply_phi(s.h, truth, clean)
            sigma = inputs.sigma_for_snr(clean, snr_db)
            Y = (clean + inputs.complex_noise(M, sigma, seed + 101 * c)).astype(np.complex64)
            B.ps_set_visibilities(s.h, Y)
            dirty = np.empty((4, n, n), np.float32)
            B.ps_apply_phi_adjoint(s.h, Y, dirty)
            s.set_state({"S": dirty})
            gamma = gamma_factor * B.ps_max_abs_analysis(s.h) / B.ps_get_params(s.h)["opnorm_sq"]
        eps = np.array([chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(nblocks)])
        out.append(Problem(n, levels, uv, Y, w, off, eps, gamma))
    return out


SIZE_MIX = ((64, 0.4), (128, 0.3), (256, 0.2), (512, 0.1))
# The served stream adds a share of large jobs to that mix: 1024^2 images with M uniform in
# [200k, 2M] rows, 5 % of the requests.
LARGE_JOBS = (1024, 0.05, (200_000, 2_000_000))


def request_stream(rate: float, duration: float, seed: int, pool: list[Problem],
                   large_pool: list[Problem] | None = None, large_share: float = 0.0) -> list[tuple[float, Problem]]:
    """Poisson arrivals at `rate` per second over `duration` seconds, each a draw from `pool`,
    or with probability `large_share` from `large_pool`."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        if large_pool and rng.random() < large_share:
            out.append((t, large_pool[int(rng.integers(len(large_pool)))]))
        else:
            out.append((t, pool[int(rng.integers(len(pool)))]))
