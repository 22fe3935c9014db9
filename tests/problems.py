"""Seeded test problems shared by the GPU parity tests.

Inputs come from paper_1801_02417_gb300.inputs; clean visibilities come from the
oracle's direct-DFT phi (never from the CUDA path). Every array handed to the
CUDA library is rounded to its storage precision first (float64 uv, float32
weights, complex64 visibilities) and the oracle receives the same rounded values.
"""
import numpy as np

from oracle import measurement as meas
from oracle import primal_dual as opd
from paper_1801_02417_gb300 import inputs


def make_problem(n, M, levels, nblocks, seed=1, snr=30.0, omega=None, coverage="tracks", weight_spread=0.3,
                 stations=8, n_compact=0):
    if coverage == "tracks":
        dumps = max(8, int(np.ceil(M / (stations * (stations - 1) / 2))) + 2)
        wl = inputs.Workload("test", n, M, stations, dumps, levels, nblocks, 0, 0, snr, n_compact, seed)
        uv = inputs.uv_coverage(wl, omega_max=omega or inputs.EHT_OMEGA_MAX)
    else:
        uv = inputs.random_uv(M, seed, omega or 0.9 * np.pi)
    w = inputs.visibility_weights(M, seed, weight_spread).astype(np.float32)
    truth = inputs.stokes_source(n, seed, n_compact)
    clean = meas.phi(truth, uv, w.astype(np.float64))
    sigma = inputs.sigma_for_snr(clean, snr)
    Y = (clean + inputs.complex_noise(M, sigma, seed)).astype(np.complex64)
    off = inputs.block_offsets(M, nblocks)
    eps = np.array([meas.chi2_epsilon(int(off[b + 1] - off[b]), sigma) for b in range(nblocks)])
    prob = opd.Problem(n, levels, uv, w.astype(np.float64), Y.astype(np.complex128), off, eps)
    return {"uv": uv, "w": w, "Y": Y, "off": off, "eps": eps, "truth": truth, "sigma": sigma, "prob": prob}


def rel_err(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
