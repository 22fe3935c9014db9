"""Write the FP64 oracle's full solve of the 256 x 256 workload to img256_m50k_solve.npz.

The workload: 256^2 Stokes I, Q, U, V, M = 50,000 rows from 10 stations, 8 l2
blocks, 4 wavelet levels, 500 iterations with 5 reweights (Algorithm 2 with the
NNLS start of Section 4.3.4: 6 cycles of 83 iterations, the first in NNLS mode).
The direct-DFT oracle needs ~5 s per iteration at this size, so its result is
stored once rather than recomputed by every GPU test run. Only `oracle/` and the
seeded input generators run here; nothing comes from the CUDA path.

Stored: the final maps S (FP64), the oracle's ||phi||^2 (ARPACK Lanczos) and the
step sizes and gamma of the solve, per-block residual norms ||phi(S) - Y||, the
violation threshold zeta and N_p at zeta and at 0, and checksums of the inputs so
that a test can confirm it regenerated the same problem.

    python tests/golden/make_img256_solve.py      # ~45 min on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import measurement as meas  # noqa: E402
from oracle import primal_dual as opd  # noqa: E402
from oracle import wavelets as wav  # noqa: E402
from paper_1801_02417_gb300 import inputs  # noqa: E402
from problems import input_checksums, make_problem  # noqa: E402

OUT = os.path.join(HERE, "img256_m50k_solve.npz")


def main() -> None:
    wl = inputs.WORKLOADS["img256_m50k"]
    t0 = time.time()
    pb = make_problem(wl.n, wl.M, wl.levels, wl.nblocks, seed=wl.seed, stations=wl.stations,
                      weight_spread=0.0)
    prob = pb["prob"]
    on = meas.op_norm_sq_lanczos(pb["uv"], prob.w, wl.n)
    print(f"||phi||^2 = {on:.9e}  ({time.time() - t0:.0f} s)", flush=True)
    dirty = meas.phi_adjoint(prob.Y, pb["uv"], prob.w, wl.n)
    gamma = 1e-3 * float(np.max(np.abs(wav.psi_adjoint(dirty, wl.levels)))) / on
    ref = opd.solve(prob, wl.iterations, wl.reweights, gamma, on)
    S = ref["S"]
    print(f"solve done ({time.time() - t0:.0f} s)", flush=True)
    res = opd.residual_norms(S, prob)
    zeta = opd.zeta_threshold(S, prob, 3.0)
    p = opd.step_sizes(on, opd.POLARIZED)
    np.savez_compressed(
        OUT, S=S, opnorm_sq=on, gamma=gamma, tau=p.tau, rho1=p.rho1, rho2=p.rho2, rho3=p.rho3,
        iterations=wl.iterations, reweights=wl.reweights, block_residual=res, eps=pb["eps"],
        zeta=zeta, violations=opd.violation_count(S, zeta), violations_raw=opd.violation_count(S, 0.0),
        **input_checksums(pb))
    print(f"wrote {OUT}: residual/eps = {np.round(res / pb['eps'], 4)}, zeta = {zeta:.3e}, "
          f"N_p = {opd.violation_count(S, zeta)} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
