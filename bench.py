"""Throughput of the Polarized SARA primal-dual iteration on GB300.

One step = one iteration of Algorithm 1 (every hot-path stage: primal/epigraph
sweep, SARA analysis + soft-threshold dual, SARA synthesis, NUFFT forward +
degrid + l2-ball dual, gridding + adjoint NUFFT) on the 1024x1024 4-Stokes,
2,000,000-visibility, 32-block, 6-level workload, with inputs resident in HBM.

Prints one JSON line. --impl reference times the FP64 CPU oracle instead (the
reference arm of this benchmark), on bounded samples of the same workload.
Multi-GPU: independent replicas, one per rank (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1801_02417_gb300 import inputs  # noqa: E402

METRIC = "PD iters/s at 1024² 4-Stokes 2M vis"
WORKLOAD = "img1024_m2m"


def chi2_epsilon(M_b: int, sigma: float) -> float:
    """eps^2 = (8M + 2 sqrt(16M)) sigma^2 / 2 (Section 5.1)."""
    dof = 8.0 * M_b
    return math.sqrt((dof + 2.0 * math.sqrt(2.0 * dof)) * sigma * sigma / 2.0)


def make_inputs(wl):
    uv = inputs.uv_coverage(wl)
    w = inputs.visibility_weights(wl.M, wl.seed, 0.0).astype(np.float32)
    truth = inputs.stokes_source(wl.n, wl.seed, wl.n_compact).astype(np.float32)
    off = inputs.block_offsets(wl.M, wl.nblocks)
    return uv, w, truth, off


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline model
def stage_bytes(n: int, L: int, M: int, Wd: int) -> dict:
    """Algorithmic DRAM bytes of each stage of one iteration (each array read/written once).

    Per map and basis the level-l details are 3 N / 4^l coefficients and the level-l
    approximation N / 4^l; the 8 bases x 4 maps give 24 N detail coefficients at level 1
    and 8 N below it. The analysis epilogue reads A and gamma W and writes A (12 B per
    coefficient); the synthesis reads A (4 B)."""
    N = n * n
    approx = sum(32 * 4 * (N >> (2 * l)) for l in range(1, L))       # 32 (map, basis) approximations
    a1 = 32 * 4 * (N >> 2) if L > 1 else 0                            # level-1 approximations
    return {
        "primal": 192 * N,                          # S,C (16+16), Z,D (8+8), PsiA, Adj, A0, T0 read; S,Xb,Z,C,D,A0 written
        "analysis": 16 * N + 12 * 24 * N + a1,      # Xb read; level-1 details A r/w + T read; approximations written
        "analysis_coarse": 12 * 8 * N + 2 * approx - a1,   # coarser coefficients; approximations read and written
        "synthesis_coarse": 4 * 8 * N + 2 * approx - a1,   # coarser coefficients; approximations written and read
        "synthesis": 4 * 24 * N + a1 + 16 * N + 16 * N,    # level-1 details, approximations, A0 read; PsiA written
        "fwd_fft": 16 * N + 2 * 16 * n * Wd + 16 * Wd * Wd,
        "degrid": M * (16 + 32 + 32 + 32) + 16 * Wd * Wd,   # rec, R r/w, Y; spectrum window once
        "ball": 0,
        "grid": M * (16 + 32) + 2 * 32 * Wd * Wd,      # rec, R; accumulator clear + write
        "adj_fft": 32 * Wd * Wd + 2 * 16 * n * Wd + 16 * N,
    }


def model_bytes(n: int, M: int) -> dict:
    """The byte model of the path (each state array read and written once, read-only inputs
    read once, X^bar and the wavelet pyramid kept on chip by fusion, the NUFFT grids at the
    minimum two-pass FFT): 912 N + 108 M per iteration, and the share of each single-kernel
    stage under it. Level 1 of the analysis holds 24 N of the 36 N coefficients (A read and
    written, gamma W read: 12 B each); the primal sweep reads and writes S, Z, C, D and the Dirac
    coefficients (with their thresholds)."""
    N = n * n
    return {"iteration": 912 * N + 108 * M, "analysis": 12 * 24 * N, "primal": 96 * N + 12 * 4 * N}


def stage_flops(n: int, M: int, W: int = 7) -> dict:
    """Algorithmic FP32 FLOPs of the stages with a compute ceiling (2 per FMA). One level of one
    basis of filter length LF over an m x m map costs 2 m^2 LF FMAs (rows, then columns, in the
    polyphase form) in either direction, and the bases' lengths sum to 72 (db1..db8: 2..16):
    1152 N at the finest level over 4 maps, plus the step-6 update (an FMA per level-1 detail).
    Degridding: W^2 taps x 2 spectrum positions x 4 real FMAs per row, plus the mixing and the
    dual update; gridding the mirror."""
    N = n * n
    return {"analysis": 1152 * N + 2 * 24 * N, "synthesis": 1152 * N + 8 * N,
            "degrid": M * (W * W * 2 * 8 + 96), "grid": M * (W * W * 2 * 8 + 48)}


# Stages that are a single kernel launch per iteration, and that kernel's name in ncu.
SINGLE_KERNEL_STAGES = {"primal": "k_primal", "analysis": "k_ana_l1", "synthesis": "k_syn2_fine",
                        "degrid": "k_degrid", "grid": "k_grid"}


def stage_kernel(stage: str, tuning: list) -> str:
    """Name of the kernel a single-kernel stage launches under the handle's launch choices."""
    if stage == "analysis" and tuning[3] == 1:
        return "k_ana_pers"
    if stage == "analysis" and tuning[3] >= 2:
        return "k_ana_l1m"
    if stage == "synthesis" and tuning[0] == 2:
        return "k_syn2_fine_pers"
    return SINGLE_KERNEL_STAGES[stage]


def kernel_sources_digest() -> str:
    """SHA-256 of the CUDA sources: DRAM counters taken from another build are not reported."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1801_02417_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def dram_traffic(kernel: str, workload: str):
    """dram__bytes_read.sum + dram__bytes_write.sum of one launch of `kernel`, from the committed
    ncu summary of this workload, or None when absent or taken from other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None, None
    if rec.get("sources_sha256") != kernel_sources_digest():
        return None, os.path.relpath(path, ROOT) + " (stale: kernels changed)"
    k = rec.get("kernels", {}).get(kernel)
    return (None if k is None else k["bytes_per_launch"]), os.path.relpath(path, ROOT)


def window_side(uv: np.ndarray, n: int, W: int = 7) -> int:
    K = 2 * n
    c = np.floor(np.abs(uv) * K / (2 * np.pi) + 0.5).max() if len(uv) else 0
    R = int(c) + W // 2 + 1
    return 2 * R + 1 if 2 * R + 1 <= K else K


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(n: int, L: int, uv: np.ndarray, w: np.ndarray, M: int, budget_s: float, seed: int = 0) -> dict:
    """Seconds per full oracle iteration of Algorithm 1 at (n, L, M), extrapolated from samples.

    Times, as the oracle runs them: the per-pixel steps on the full maps (once);
    the analysis + synthesis of a few (map, basis) pairs (each of the 32 pairs
    costs the same); phi + phi^dagger on a subset of rows (cost linear in rows).
    """
    from oracle import measurement as meas
    from oracle import prox
    from oracle import wavelets as wav

    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    S = rng.normal(size=(4, n, n))
    Z = rng.normal(size=(2, n, n))
    C = rng.normal(size=(4, n, n))
    D = rng.normal(size=(2, n, n))
    A0 = rng.normal(size=(4, n, n))
    # Per-pixel part (steps 3-4, 9-12, Dirac of 5-6).
    t = time.perf_counter()
    X = S - 0.33 * (A0 + C)
    Z1 = prox.proj_V(Z - 0.33 * D)
    Sb, Zb = 2 * X - S, 2 * Z1 - Z
    Ct, Dt = C + Sb, D + Zb
    prox.proj_E1(Ct[0], Dt[0])
    prox.proj_E2(Ct[1:4], Dt[1])
    prox.soft_threshold(A0 + Sb / 3, np.abs(A0))
    t_pix = time.perf_counter() - t
    # Wavelet pairs.
    pairs = []
    x = rng.normal(size=(n, n))
    b = 1
    while True:
        t = time.perf_counter()
        c = wav.dwt2(x, wav.FILTERS[b], L)
        wav.idwt2(c, wav.FILTERS[b], L)
        prox.soft_threshold(c, np.abs(c))
        pairs.append(time.perf_counter() - t)
        b = b % 8 + 1
        if len(pairs) >= 8 or time.perf_counter() - t0 > 0.6 * budget_s:
            break
    t_pairs = 32 * statistics.mean(pairs)
    # phi + phi^dagger on a row subset.
    rows = 64
    sub = rng.choice(len(uv), size=min(rows, len(uv)), replace=False)
    Sm = rng.normal(size=(4, n, n))
    t = time.perf_counter()
    Bv = meas.phi(Sm, uv[sub], w[sub])
    meas.phi_adjoint(Bv, uv[sub], w[sub], n)
    t_rows = time.perf_counter() - t
    t_vis = t_rows * M / len(sub)
    total = t_pix + t_pairs + t_vis
    return {"seconds_per_iter": total, "t_pixels": t_pix, "t_wavelets": t_pairs, "t_phi": t_vis,
            "pairs_timed": len(pairs), "rows_timed": int(len(sub)), "wall": time.perf_counter() - t0}


def cpu_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count() or 1


# ------------------------------------------------------------------ batched and served
def draw_requests(count: int, seed: int, large: bool = False):
    """Independent problems of the batched workload: sizes 64/128/256/512 with weights
    0.4/0.3/0.2/0.1, M uniform in [2k, 200k], input SNR uniform in [20, 40] dB, 4 levels.
    large=True: the served stream's large jobs instead, 1024^2 with M uniform in [200k, 2M]."""
    from paper_1801_02417_gb300.serve import LARGE_JOBS, SIZE_MIX, synthesize_problem
    rng = np.random.default_rng(seed)
    sizes = [n for n, _ in SIZE_MIX]
    probs = [p for _, p in SIZE_MIX]
    out = []
    for i in range(count):
        if large:
            n, (m0, m1) = LARGE_JOBS[0], LARGE_JOBS[2]
        else:
            n, (m0, m1) = int(rng.choice(sizes, p=probs)), (2000, 200000)
        M = int(rng.integers(m0, m1 + 1))
        nb = 1 if M < 50000 else (4 if M < 500000 else 32)
        out.append(synthesize_problem(n, 4, M, seed + 100 + i, nb, snr_db=float(rng.uniform(20, 40))))
    return out


def batched_measure(problems, iterations: int = 500, reweights: int = 5) -> dict:
    """Whole Algorithm 2 solves (NNLS start, `reweights` reweighted cycles, `iterations` in
    all) of every problem: the batched path (every cycle advances all problems by one batch
    graph launch per iteration, solver.solve_batched) against the same solves one after
    another on the plain single-solve path. Launch choices from the autotuner, one run per
    size class, for both."""
    from paper_1801_02417_gb300.serve import apply_tuning
    from paper_1801_02417_gb300.solver import PolarizedSARA, Schedule, solve_batched

    def start(p):
        s = PolarizedSARA(p.n, p.levels)
        s.set_measurements(p.uv, p.vis, p.weights, p.offsets, p.eps)
        apply_tuning(s, p.n, p.uv.shape[0], cache)
        return s
    cache = {}
    schedules = [Schedule(iterations, reweights, p.gamma) for p in problems]
    # Preparation (handles, row sort, operator norm, tuning) is outside both timings.
    seq = 0.0
    for p, sch in zip(problems, schedules):
        with start(p) as s:
            s.synchronize()
            t = time.perf_counter()
            s.solve(sch)
            s.synchronize()
            seq += time.perf_counter() - t
    ss = [start(p) for p in problems]
    try:
        for s in ss:
            s.synchronize()
        t = time.perf_counter()
        solve_batched(ss, schedules)
        bat = time.perf_counter() - t
    finally:
        for s in ss:
            s.close()
    k = len(problems)
    return {"problems": k, "iterations": iterations, "reweights": reweights,
            "sizes": {str(n): sum(p.n == n for p in problems) for n in sorted({p.n for p in problems})},
            "tuning": {f"n{key[0]}_M<2^{key[1]}": v for key, v in sorted(cache.items())},
            "batched_s": bat, "sequential_s": seq, "speedup": seq / bat,
            "solves_per_s_batched": k / bat, "solves_per_s_sequential": k / seq,
            "solve_iters_per_s_batched": k * iterations / bat, "solve_iters_per_s_sequential": k * iterations / seq}


def default_gamma(s, dirty: np.ndarray, factor: float = 1e-3) -> float:
    """gamma = factor * max |Psi^dagger phi^dagger Y| / ||phi||^2: the dirty image's analysis
    coefficients brought back to image units (phi^dagger phi has peak ||phi||^2). gamma leaves
    the minimiser unchanged and sets how fast the duals balance; in back-projected units it
    would exceed the data dual's scale by ~||phi||^2 and stall the data fit."""
    from paper_1801_02417_gb300 import binding as B
    on = B.ps_get_params(s.h)["opnorm_sq"]
    return factor * float(np.max(np.abs(s.psi_adjoint(dirty)))) / on


def small_configs(iters: int = 500) -> dict:
    """Iteration rate of the small workloads (64^2 / 2,000 rows and 256^2 / 50,000 rows) on
    the same launch path (autotuned choices, multi-iteration graphs), timed with CUDA events on
    the handle's stream; at these sizes an iteration is a chain of short kernels, so the rate
    measures launch and dependency latency more than bandwidth."""
    import torch
    from paper_1801_02417_gb300 import binding as B
    from paper_1801_02417_gb300.solver import PolarizedSARA
    out = {}
    stream = torch.cuda.Stream()
    for name in ("img64_m2k", "img256_m50k"):
        wl = inputs.WORKLOADS[name]
        uv, w, truth, off = make_inputs(wl)
        with PolarizedSARA(wl.n, wl.levels, stream=stream.cuda_stream) as s:
            s.set_measurements(uv, np.zeros((wl.M, 4), np.complex64), w, off, np.ones(wl.nblocks))
            clean = np.empty((wl.M, 4), np.complex64)
            B.ps_apply_phi(s.h, truth, clean)
            sigma = inputs.sigma_for_snr(clean, wl.snr_db)
            Y = (clean + inputs.complex_noise(wl.M, sigma, wl.seed)).astype(np.complex64)
            eps = np.array([chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(wl.nblocks)])
            s.set_measurements(uv, Y, w, off, eps)
            s.set_sara_weights(None, 0.0)
            s.set_mode(B.PS_POLARIZED)
            picks = B.ps_autotune(s.h, reps=5)
            s.pd_iterate(16)
            s.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s.pd_iterate(iters)
            ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1) / iters
            stages = B.ps_profile_stages(s.h, 50)
            out[name] = {"iters_per_s": 1000.0 / ms, "us_per_iter": 1000.0 * ms, "iterations_timed": iters,
                         "kernels_per_iteration": B.ps_kernels_per_iteration(s.h),
                         "stages_us_sum": 1000.0 * sum(stages.values()),
                         "tuning": {k: v[0] for k, v in picks.items() if not k.startswith("reserved")}}
    return out


def np_comparison(wl_name: str = "img256_m50k", iterations: int = 0, reweights: int = -1) -> dict:
    """Section 5.2 protocol on synthetic data: the same schedule (NNLS start, reweighted cycles;
    the workload's own budget unless given) with and without the polarization constraint;
    N_p = pixels with -I + ||(Q,U,V)|| > zeta, reported beside the data fit reached."""
    from paper_1801_02417_gb300 import binding as B
    from paper_1801_02417_gb300.solver import PolarizedSARA, Schedule
    wl = inputs.WORKLOADS[wl_name]
    iterations = iterations or wl.iterations
    reweights = wl.reweights if reweights < 0 else reweights
    uv, w, truth, off = make_inputs(wl)
    out = {"workload": wl.name, "iterations": iterations, "reweights": reweights}
    with PolarizedSARA(wl.n, wl.levels) as s:
        s.set_measurements(uv, np.zeros((wl.M, 4), np.complex64), w, off, np.ones(wl.nblocks))
        clean = np.empty((wl.M, 4), np.complex64)
        B.ps_apply_phi(s.h, truth, clean)
        sigma = inputs.sigma_for_snr(clean, wl.snr_db)
        Y = (clean + inputs.complex_noise(wl.M, sigma, wl.seed)).astype(np.complex64)
        eps = np.array([chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(wl.nblocks)])
        s.set_measurements(uv, Y, w, off, eps)
        dirty = np.empty((4, wl.n, wl.n), np.float32)
        B.ps_apply_phi_adjoint(s.h, Y, dirty)
        gamma = default_gamma(s, dirty)
        for name, mode in (("polarized", B.PS_POLARIZED), ("soc", B.PS_SOC), ("no_constraint", B.PS_NO_CONSTRAINT)):
            s.set_measurements(uv, Y, w, off, eps)      # fresh state
            t = time.perf_counter()
            S = s.solve(Schedule(iterations, reweights, gamma), mode=mode)
            st = s.stats()
            out[name] = {"N_p": int(st["violations"]), "N_p_zeta0": int(st["violations_raw"]),
                         "zeta": st["zeta"], "rel_l2_vs_truth": float(np.linalg.norm(S - truth) / np.linalg.norm(truth)),
                         "max_block_residual_over_eps": float(np.max(st["block_residual"] / eps)),
                         "solve_s": time.perf_counter() - t}
        # The TV problems of Algorithm 3 (Table 2's TV and l1 + TV columns) with and without
        # the constraint, same iteration budget (Algorithm 3 has no reweighting). Weights in
        # the data term's units: 1e-2 of the largest gradient (TV) or value (l1) of the
        # Stokes-domain dirty image phi~^dagger Y~ = phi^dagger Y / 2, the same for all maps
        # (the paper tunes them per map for the lowest NRMSE).
        gxy = np.stack([np.roll(dirty, -1, axis=-1) - dirty, np.roll(dirty, -1, axis=-2) - dirty])
        mu = 1e-2 * float(np.abs(gxy).max()) / 2.0
        nu = 1e-2 * float(np.abs(dirty).max()) / 2.0
        for name, mode in (("tv", B.PS_TV), ("tv_no_constraint", B.PS_TV_NC), ("l1tv", B.PS_L1TV),
                           ("l1tv_no_constraint", B.PS_L1TV_NC)):
            s.set_measurements(uv, Y, w, off, eps)
            s.set_mode(mode)
            B.ps_set_tv_weights(s.h, [mu] * 4, [nu] * 4)
            t = time.perf_counter()
            s.pd_iterate(iterations)
            S = s.get_stokes()
            st = s.stats()
            out[name] = {"N_p": int(st["violations"]), "N_p_zeta0": int(st["violations_raw"]),
                         "zeta": st["zeta"], "rel_l2_vs_truth": float(np.linalg.norm(S - truth) / np.linalg.norm(truth)),
                         "max_block_residual_over_eps": float(np.max(st["block_residual"] / eps)),
                         "solve_s": time.perf_counter() - t}
        s.set_mode(B.PS_POLARIZED)
    return out


def served_measure(pool, large_pool, rate: float, duration: float, seed: int, solo_seconds: float) -> dict:
    """The served stream: Poisson arrivals at `rate`/s for `duration` s drawn from the batched
    mix plus a 5 % share of large (1024^2) jobs, each solved to a relative change of I, Q, U of
    1e-4 per cycle (Eq. stop_crit as printed, <= 2000 iterations, 5 reweights), admitted by device footprint,
    state resident, overlapping on the device (continuous batching). The one-at-a-time path
    serves the first `solo_seconds` of the same arrivals (a bounded sample: it falls behind the
    arrival rate, so its queue, and its latencies, grow with the window)."""
    from paper_1801_02417_gb300.serve import LARGE_JOBS, Policy, Server, request_stream, summarize
    reqs = request_stream(rate, duration, seed, pool, large_pool, LARGE_JOBS[1])
    pol = Policy(rule="rel", rel_tol=1e-4, maps=3, max_iter=2000, reweights=5, check_every=20)
    t0 = time.perf_counter()
    res = Server(hbm_budget=64 << 30, max_active=32, policy=pol).run(reqs)
    wall = time.perf_counter() - t0
    cont = summarize(res)
    big = [r for r in res if reqs[r.rid][1].n == LARGE_JOBS[0]]
    cont["large_jobs"] = summarize(big) if big else {"solves": 0}
    solo_reqs = [r for r in reqs if r[0] <= solo_seconds]
    solo = summarize(Server(hbm_budget=64 << 30, max_active=1, policy=pol).run(solo_reqs))
    solo["window_s"] = solo_seconds
    return {"rate_per_s": rate, "duration_s": duration, "requests": len(reqs),
            "large_share": LARGE_JOBS[1], "large_requests": sum(1 for _, p in reqs if p.n == LARGE_JOBS[0]),
            "rule": "relative change of I, Q, U <= 1e-4 per cycle (Eq. stop_crit as printed)", "wall_s": wall,
            "continuous_batching": cont, "one_at_a_time": solo}


def hyperspectral_measure(nchan: int = 8, n: int = 256, M: int = 50000, seed: int = 0) -> dict:
    """Multi-frequency observation (20% bandwidth, spectral index -0.7, Faraday rotation):
    one independent Polarized SARA solve per channel, all channels submitted at once to the
    continuous-batching server (each on its own stream, overlapping) vs one after another."""
    from paper_1801_02417_gb300.serve import Policy, Server, summarize, synthesize_channels
    chans = synthesize_channels(n, 4, M, nchan, seed, nblocks=8)
    pol = Policy(rule="rel", rel_tol=1e-4, maps=3, max_iter=2000, reweights=5, check_every=20)
    reqs = [(0.0, p) for p in chans]
    t0 = time.perf_counter()
    cont = Server(hbm_budget=64 << 30, max_active=nchan, policy=pol).run(reqs)
    t_cont = time.perf_counter() - t0
    t0 = time.perf_counter()
    Server(hbm_budget=64 << 30, max_active=1, policy=pol).run(reqs)
    t_seq = time.perf_counter() - t0
    s = summarize(cont)
    return {"channels": nchan, "n": n, "rows_per_channel": M, "frac_bandwidth": 0.2,
            "batched_s": t_cont, "sequential_s": t_seq, "speedup": t_seq / t_cont,
            "channels_per_s": nchan / t_cont, "iterations_mean": s["iterations_mean"]}


# ------------------------------------------------------------------ arms
def aggregate_replicas(ms: float, steps: int, world: int, device: str = "cuda"):
    """Replicas (one independent solve per rank, no collective on the data path): the job's
    time is the slowest rank's timed region, and the job processed world x steps iterations.
    Returns (max ms over ranks, whole-job iterations/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1000.0)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args) -> None:
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = inputs.WORKLOADS[args.workload]
    uv, w, truth, off = make_inputs(wl)
    per_step_budget = max(0.5, 150.0 / max(1, args.steps + args.warmup))
    samples = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(wl.n, wl.levels, uv, w.astype(np.float64), wl.M, per_step_budget, seed=i)
        if i >= args.warmup:
            samples.append(r["seconds_per_iter"])
    sec = statistics.mean(samples)
    value = 1.0 / sec
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "M": wl.M, "blocks": wl.nblocks, "levels": wl.levels},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: FP64 oracle per-pixel steps on full 1024^2 maps, analysis+synthesis "
                                   "of sampled (map, basis) pairs x32, phi+phi^dagger on 64 rows scaled to 2M"},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_own(args) -> None:
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1801_02417_gb300 import _build
    from paper_1801_02417_gb300 import binding as B
    from paper_1801_02417_gb300.solver import PolarizedSARA
    if rank == 0 or not os.path.exists(_build.LIB):
        _build.build_library()
    if world > 1:
        dist.barrier()
    B.lib()

    wl = inputs.WORKLOADS[args.workload]
    n, L, M = wl.n, wl.levels, wl.M
    uv, w, truth, off = make_inputs(wl)
    # A dedicated stream: the handle launches on it and the CUDA events below are
    # recorded on it (torch's default stream would be handle 0 = "create your own").
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = PolarizedSARA(n, L, stream=stream.cuda_stream)
    # Clean visibilities from the library's own phi, then noise at the input SNR.
    zeros = np.zeros((M, 4), np.complex64)
    eps1 = np.ones(wl.nblocks)
    s.set_measurements(uv, zeros, w, off, eps1)
    clean = np.empty((M, 4), np.complex64)
    B.ps_apply_phi(s.h, truth, clean)
    sigma = inputs.sigma_for_snr(clean, wl.snr_db)
    Y = (clean + inputs.complex_noise(M, sigma, wl.seed)).astype(np.complex64)
    eps = np.array([chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(wl.nblocks)])
    s.set_measurements(uv, Y, w, off, eps)
    dirty = np.empty((4, n, n), np.float32)
    B.ps_apply_phi_adjoint(s.h, Y, dirty)
    gamma = default_gamma(s, dirty)
    s.set_sara_weights(None, gamma)
    s.set_mode(B.PS_POLARIZED)
    # Launch choices measured on this problem before the warm-up (or forced by --tuning,
    # e.g. to profile the configuration the autotuner picks without a profiler attached).
    if args.tuning:
        B.ps_set_tuning(s.h, [int(v) for v in args.tuning.split(",")])
        tuning = dict(zip(B.TUNE_SLOTS, B.ps_get_tuning(s.h)))
    else:
        picks = B.ps_autotune(s.h, reps=5)
        tuning = {k: v[0] for k, v in picks.items() if not k.startswith("reserved")}

    # Warm-up, then exactly K timed steps between barriers.
    s.pd_iterate(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()        # ncu --profile-from-start off captures only this region
    ev0.record(stream)
    s.pd_iterate(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms, value = aggregate_replicas(ms, args.steps, world, "cuda")
    ms_per_step = ms / args.steps
    launches = B.ps_kernels_per_iteration(s.h) * args.steps

    # Stage timing (CUDA events between stages, same launch configuration, eager).
    prof_iters = min(args.steps, 20)
    stages = B.ps_profile_stages(s.h, prof_iters)
    Wd = window_side(uv, n)
    sbytes = stage_bytes(n, L, M, Wd)
    mbytes = model_bytes(n, M)
    sflops = stage_flops(n, M)
    # Dominant kernel: the slowest stage that is one kernel launch per iteration. Its bytes are
    # the byte model's share where the model assigns one (the level-1 analysis: A read and
    # written, gamma W read), else every array it touches once.
    dom = max(SINGLE_KERNEL_STAGES, key=lambda k: stages[k])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dom_bytes = mbytes.get(dom, sbytes[dom])
    achieved = dom_bytes / (stages[dom] * 1e-3) / 1e9
    dom_kernel = stage_kernel(dom, B.ps_get_tuning(s.h))
    traffic, traffic_src = dram_traffic(dom_kernel, wl.name)
    total_bytes = sum(sbytes.values())
    fp32 = {"packed_flops": B.ps_fp32_peak(True), "scalar_flops": B.ps_fp32_peak(False)}
    fp32_peak = max(fp32["packed_flops"], fp32["scalar_flops"])

    # End to end through the C ABI with host buffers (pinned), as a user runs a solve:
    # upload of the measurements (row sort, operator-norm estimate), then per step one
    # iteration and a device->host read of its stopping metric (the per-map relative
    # change of Eq. stop_crit: 8 FP64 sums and the device flags), and the Stokes maps read
    # back once at the end. The metric of iteration k is requested after it and read while
    # iteration k + 1 runs (ps_rel_change_request / ps_rel_change_result), so the host's
    # stopping decision does not idle the GPU; the synchronous read (ps_get_rel_change after
    # every iteration) is timed beside it.
    e2e = None
    if rank == 0 and not args.kernels_only:
        uv_p = torch.from_numpy(uv).pin_memory()
        Y_p = torch.from_numpy(Y.view(np.float32)).pin_memory()
        w_p = torch.from_numpy(w).pin_memory()
        out_p = torch.empty((4, n, n), dtype=torch.float32).pin_memory()
        ke = wl.iterations                              # one solve of the workload's length (1,000 iterations)
        d2h_metric = 8 * 8 + 4 * 4                      # relative-change sums and device flags per step
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.ps_set_measurements(s.h, uv_p, Y_p, w_p, off, eps)
        s.set_sara_weights(None, gamma)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        s.pd_iterate(1)
        B.ps_rel_change_request(s.h)
        for _ in range(ke - 1):
            s.pd_iterate(1)
            B.ps_rel_change_result(s.h)                 # the previous iteration's metric
            B.ps_rel_change_request(s.h)
        B.ps_rel_change_result(s.h)
        B.ps_get_stokes(s.h, out_p)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = uv.nbytes + Y.nbytes + w.nbytes
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for _ in range(ke):
            s.pd_iterate(1)
            B.ps_get_rel_change(s.h)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t2
        # The stricter variant: the full Stokes maps read back after every iteration.
        km = min(ke, 20)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(km):
            s.pd_iterate(1)
            B.ps_get_stokes(s.h, out_p)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t1
        e2e = {"value": ke / te, "unit": "iter/s", "h2d_bytes_per_step": int(h2d / ke),
               "d2h_bytes_per_step": int(d2h_metric + out_p.numel() * 4 / ke),
               "solve_iterations": ke, "setup_s": t_setup, "steps_only_value": ke / (te - t_setup),
               "note": f"one {ke}-iteration solve through the C ABI from pinned host buffers: measurements uploaded "
                       "once (row sort, operator-norm estimate, default gamma: setup_s), then per step one iteration "
                       "+ read of its relative-change metric (requested after the iteration, read while the next "
                       "one runs); Stokes maps read once at the end",
               "synchronous_read": {"steps_only_value": ke / ts, "unit": "iter/s",
                                    "note": "ps_get_rel_change (synchronising) after every iteration"},
               "maps_every_step": {"value": km / tm, "unit": "iter/s", "d2h_bytes_per_step": int(out_p.numel() * 4)}}

    # The direct cone-dual variant (PS_SOC: no Z, D) on the same problem and launch path.
    soc = None
    if rank == 0 and not args.kernels_only:
        s.set_mode(B.PS_SOC)
        s.pd_iterate(args.warmup)
        torch.cuda.synchronize()
        ev0.record(stream)
        s.pd_iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_soc = ev0.elapsed_time(ev1) / args.steps
        soc = {"iters_per_s": 1000.0 / ms_soc, "ms_per_step": ms_soc,
               "algorithmic_bytes": total_bytes - 32 * n * n,
               "note": "PS_SOC: polarization cone as one dual (no Z, D), same problem as the epigraph split"}
        s.set_mode(B.PS_POLARIZED)

    # The TV problem with the constraint (Algorithm 3) on the same data and launch path:
    # the gradient step replaces the data dual, grad replaces the SARA dictionary.
    tvv = None
    if rank == 0 and not args.kernels_only:
        B.ps_set_tv_weights(s.h, [1e-3 * gamma * 3.0] * 4)
        s.set_mode(B.PS_TV)
        s.pd_iterate(args.warmup)
        torch.cuda.synchronize()
        ev0.record(stream)
        s.pd_iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_tv = ev0.elapsed_time(ev1) / args.steps
        tvv = {"iters_per_s": 1000.0 / ms_tv, "ms_per_step": ms_tv,
               "kernels_per_iteration": B.ps_kernels_per_iteration(s.h),
               "note": "PS_TV: Algorithm 3 (TV prior, gradient step on the data term, polarization "
                       "constraint by the epigraph split) on the same measurements"}
        s.set_mode(B.PS_POLARIZED)

    batched = served = np_cmp = hyper = small = None
    if rank == 0 and world == 1 and not args.no_serve and not args.kernels_only:
        small = small_configs()
        np_cmp = np_comparison()
        s.close()
        pool = draw_requests(args.batch, seed=wl.seed + 50)
        batched = batched_measure(pool)
        large = draw_requests(4, seed=wl.seed + 55, large=True)
        served = served_measure(pool, large, rate=args.serve_rate, duration=args.serve_seconds, seed=wl.seed + 60,
                                solo_seconds=min(args.serve_seconds, args.solo_seconds))
        hyper = hyperspectral_measure(seed=wl.seed + 70)
        s = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.kernels_only:
        r = oracle_sample(n, L, uv, w.astype(np.float64), M, budget_s=20.0)
        cpu = {"value": 1.0 / r["seconds_per_iter"], "unit": "iter/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": (f"FP64 oracle: per-pixel steps on full {n}^2 maps ({r['t_pixels']:.2f}s), "
                          f"{r['pairs_timed']} (map,basis) analysis+synthesis pairs x32/{r['pairs_timed']} "
                          f"({r['t_wavelets']:.1f}s), phi+phi^dagger on {r['rows_timed']} rows x{M // r['rows_timed']} "
                          f"({r['t_phi']:.1f}s); extrapolated per-iteration time {r['seconds_per_iter']:.1f}s")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "n": n, "stokes": 4, "M": M, "blocks": wl.nblocks, "levels": L,
                       "kernel_width": 7, "oversampling": 2, "grid_window": Wd,
                       "parallelism": "replicas" if world > 1 else "single", "tuning": tuning,
                       "l2": "no flush: per-iteration working set ~%.0f MB > 126 MB L2" % (total_bytes / 1e6),
                       "vis_iters_per_s": value * M},
            "roofline": {"bound": "hbm", "kernel": dom_kernel, "stage": dom, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": traffic_src, "peak_source": peak_src + " hbm_gbs (copy)",
                         "algorithmic_bytes": dom_bytes, "bytes_model": "byte model share" if dom in mbytes
                         else "every array touched once", "all_arrays_bytes": sbytes[dom],
                         "launch_ms": stages[dom]},
            "stage_roofline": {k: {"ms": stages[k], "algorithmic_bytes": sbytes[k],
                                   "frac": sbytes[k] / (stages[k] * 1e-3) / 1e9 / peak if stages[k] > 0 else None,
                                   **({"model_bytes": mbytes[k],
                                       "model_frac": mbytes[k] / (stages[k] * 1e-3) / 1e9 / peak} if k in mbytes
                                      else {}),
                                   **({"flops": sflops[k],
                                       "fp32_frac": sflops[k] / (stages[k] * 1e-3) / fp32_peak} if k in sflops
                                      else {})}
                               for k in stages},
            "fp32_peak": {"packed_tflops": fp32["packed_flops"] / 1e12, "scalar_tflops": fp32["scalar_flops"] / 1e12,
                          "source": "ps_fp32_peak, measured in this run (FMA chains on every SM)"},
            "iteration_roofline": {"algorithmic_bytes": mbytes["iteration"], "model": "912 N + 108 M",
                                   "achieved_gbs": mbytes["iteration"] / (ms_per_step * 1e-3) / 1e9,
                                   "frac": mbytes["iteration"] / (ms_per_step * 1e-3) / 1e9 / peak,
                                   "stage_bytes_sum": total_bytes,
                                   "stage_bytes_frac": total_bytes / (ms_per_step * 1e-3) / 1e9 / peak},
            "stages_ms": stages,
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": e2e,
            "soc_variant": soc,
            "tv_variant": tvv,
            "cpu_baseline": cpu,
            "batched": batched,
            "served": served,
            "hyperspectral": hyper,
            "np_comparison": np_cmp,
            "small_configs": small,
        }
        print(json.dumps(line), flush=True)
    if s is not None:
        s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", default="", help="force the launch choices (comma-separated PS_TUNE_* values)")
    ap.add_argument("--no-serve", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the timed iterations and the stage timing (for profiler runs)")
    ap.add_argument("--batch", type=int, default=64, help="problems in the batched measurement")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-seconds", type=float, default=120.0)
    ap.add_argument("--solo-seconds", type=float, default=15.0,
                    help="arrival window served by the one-at-a-time comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_own(args)


if __name__ == "__main__":
    main()
