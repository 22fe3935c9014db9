"""Host driver of Algorithm 2 (reweighting, Section 4.3.4) over the CUDA library.

Every step of the primal-dual iteration runs in libpolsara.so; this module only
sequences the C ABI calls: NNLS start, reweights with a decreasing delta, and the
stopping rules of Section 5.5.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Schedule:
    """Fixed budget: `iterations` split over `reweights + 1` cycles, the first in NNLS mode.

    delta^(1) = delta_factor * max |Psi^dagger S_nnls|, multiplied by delta_decay after each
    reweight (delta -> 0, Eq. weights).
    """
    iterations: int
    reweights: int
    gamma: float
    delta_factor: float = 0.1
    delta_decay: float = 0.5


class PolarizedSARA:
    """One imaging problem resident on the GPU (a ps_handle)."""

    def __init__(self, n: int, levels: int, mode: int = B.PS_POLARIZED, kernel_width: int = 7,
                 literal_ball: bool = False, tau: float = 0.0, rho1: float = 0.0, rho2: float = 0.0,
                 rho3: float = 0.0, stream=None, gamma: float = 0.0, noise_sigma: float = 0.0,
                 rel_tol: float = 0.0, resid_tol: float = 0.0, np_tol: float = 0.0, zeta_sigma: float = 0.0,
                 stop_maps: int = 0):
        """Zero for a parameter takes the library default (include/polsara.h, ps_config)."""
        cfg = B.ps_config(n=n, levels=levels, mode=mode, literal_ball=int(literal_ball),
                          kernel_width=kernel_width, stop_maps=stop_maps, tau=tau, rho1=rho1, rho2=rho2, rho3=rho3,
                          alpha=0.0, gamma=gamma, noise_sigma=noise_sigma, rel_tol=rel_tol,
                          resid_tol=resid_tol, np_tol=np_tol, zeta_sigma=zeta_sigma)
        self.n, self.levels = n, levels
        self.h = B.ps_create(cfg, stream)
        self.nblocks = 0
        self.M = 0

    def close(self) -> None:
        if self.h is not None:
            B.ps_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # Thin forwards to the C ABI.
    def set_measurements(self, uv, vis, weights, block_offsets, eps=None) -> None:
        """eps None: the chi^2 radii of Section 5.1 from the handle's noise_sigma."""
        B.ps_set_measurements(self.h, uv, vis, weights, block_offsets, eps)
        self.nblocks = len(block_offsets) - 1
        self.M = int(uv.shape[0])

    def set_sara_weights(self, W, gamma: float) -> None:
        B.ps_set_sara_weights(self.h, W, gamma)

    def get_sara_weights(self) -> np.ndarray:
        out = np.empty((4, 9, self.n, self.n), np.float32)
        B.ps_get_sara_weights(self.h, out)
        return out

    def pd_iterate(self, n_iter: int, stats: bool = False):
        """n_iter iterations; with stats=True returns the stopping-rule statistics after them."""
        return B.ps_pd_iterate(self.h, n_iter, self.nblocks if stats else None)

    def reweight(self, delta: float) -> None:
        B.ps_reweight(self.h, delta)

    def set_mode(self, mode: int) -> None:
        B.ps_set_mode(self.h, mode)

    def get_stokes(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((4, self.n, self.n), dtype=np.float32)
        B.ps_get_stokes(self.h, out)
        return out

    def get_state(self) -> dict:
        n, M = self.n, self.M
        st = {"S": np.empty((4, n, n), np.float32), "Z": np.empty((2, n, n), np.float32),
              "A": np.empty((4, 9, n, n), np.float32), "B": np.empty((M, 4), np.complex64),
              "C": np.empty((4, n, n), np.float32), "D": np.empty((2, n, n), np.float32)}
        B.ps_get_state(self.h, st)
        return st

    def set_state(self, st: dict) -> None:
        B.ps_set_state(self.h, st)

    def params(self) -> dict:
        return B.ps_get_params(self.h)

    def config(self):
        """The handle's ps_config with every default resolved (gamma: the handle's default gamma)."""
        return B.ps_get_config(self.h)

    def stats(self, zeta_sigma: float = 0.0) -> dict:
        return B.ps_compute_stats(self.h, zeta_sigma, self.nblocks)

    def synchronize(self) -> None:
        B.ps_synchronize(self.h)

    def psi_adjoint(self, S) -> np.ndarray:
        out = np.empty((4, 9, self.n, self.n), np.float32)
        B.ps_apply_psi_adjoint(self.h, S, out)
        return out

    # Algorithm 2.
    def solve(self, sch: Schedule, W0=None, mode: int = B.PS_POLARIZED) -> np.ndarray:
        """NNLS start, then `reweights` cycles of Algorithm 1 each preceded by a reweight.
        mode: PS_POLARIZED (epigraph split) or PS_SOC (direct cone dual) for the cycles."""
        per = sch.iterations // (sch.reweights + 1)
        self.set_mode(B.PS_NNLS)
        self.pd_iterate(per)
        delta = sch.delta_factor * B.ps_max_abs_analysis(self.h)
        self.set_sara_weights(W0, sch.gamma)
        self.set_mode(mode)
        for _ in range(sch.reweights):
            self.reweight(delta)
            self.pd_iterate(per)
            delta *= sch.delta_decay
        return self.get_stokes()

    def solve_until(self, gamma: float = 0.0, max_iter: int = 2000, reweights: int = 5, check_every: int = 20,
                    delta_factor: float = 0.1, delta_decay: float = 0.5, rule: str = "paper") -> dict:
        """Algorithm 2 with each cycle stopped by the rule of Section 5.5 or at the iteration cap.

        rule "paper": every criterion of Section 5.5 with the handle's tolerances (ps_config
        rel_tol, resid_tol, np_tol): the relative change of Eq. stop_crit, the data fit
        ||phi(S) - Y||_b <= (1 + vartheta) eps_b and, with the constraint, N_p <= varrho.
        rule "rel": the relative change alone (cheaper: no residual evaluation).
        The relative change covers the handle's stop_maps maps (all four by default; a map that
        stays zero counts 0).
        gamma 0 takes the handle's gamma."""
        used = 0
        per_cap = max(check_every, max_iter // (reweights + 1))
        cfg = B.ps_get_config(self.h)
        rel_tol, maps = cfg.rel_tol, cfg.stop_maps

        def cycle():
            nonlocal used
            k = 0
            while k < per_cap and used < max_iter:
                step = min(check_every, per_cap - k, max_iter - used)
                k += step
                used += step
                if rule == "paper":
                    if self.pd_iterate(step, stats=True)["converged"]:
                        break
                else:
                    self.pd_iterate(step)
                    if float(np.max(B.ps_get_rel_change(self.h)[:maps])) <= rel_tol:
                        break
        self.set_mode(B.PS_NNLS)
        cycle()
        delta = delta_factor * B.ps_max_abs_analysis(self.h)
        self.set_sara_weights(None, gamma)
        self.set_mode(B.PS_POLARIZED)
        for _ in range(reweights):
            if used >= max_iter:
                break
            self.reweight(delta)
            cycle()
            delta *= delta_decay
        return {"iterations": used, "S": self.get_stokes()}


def solve_batched(solvers: list, schedules: list, mode: int = B.PS_POLARIZED) -> list:
    """Algorithm 2 (NNLS start, reweighted cycles) for many independent problems at once.

    Every cycle advances all problems together: one launch of a batch graph (ps_batch_*)
    per iteration holds one iteration of every problem, each on its own stream, so the
    kernels of different problems overlap on the device. The schedules must share their
    iteration count and reweight count (the cycles run in lockstep); gamma and the delta
    schedule are each problem's own. Returns the Stokes maps of every problem.
    """
    shapes = {(sch.iterations, sch.reweights) for sch in schedules}
    if len(shapes) != 1 or len(schedules) != len(solvers):
        raise ValueError("solve_batched: one schedule per solver, all with the same iterations and reweights")
    iterations, reweights = shapes.pop()
    per = iterations // (reweights + 1)
    for s in solvers:
        s.set_mode(B.PS_NNLS)
    b = B.ps_batch_create([s.h for s in solvers])
    try:
        B.ps_batch_iterate(b, per)
        deltas = [sch.delta_factor * B.ps_max_abs_analysis(s.h) for s, sch in zip(solvers, schedules)]
        for s, sch in zip(solvers, schedules):
            s.set_sara_weights(None, sch.gamma)
            s.set_mode(mode)
        for _ in range(reweights):
            for s, d in zip(solvers, deltas):
                s.reweight(d)
            B.ps_batch_iterate(b, per)
            deltas = [d * sch.delta_decay for d, sch in zip(deltas, schedules)]
        B.ps_batch_synchronize(b)
    finally:
        B.ps_batch_destroy(b)
    return [s.get_stokes() for s in solvers]
