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


def input_checksums(pb):
    """Scalar summaries of a problem's inputs, stored beside oracle results so a test can confirm
    it regenerated the same problem (to rounding) before comparing against them."""
    uv = np.asarray(pb["uv"], np.float64)
    Y = np.asarray(pb["Y"], np.complex128)
    return {"chk_uv": float(np.sum(np.abs(uv))), "chk_Y": float(np.sum(np.abs(Y))),
            "chk_w": float(np.sum(np.asarray(pb["w"], np.float64))), "chk_sigma": float(pb["sigma"])}


def make_channel_problem(n, M, levels, nchan, chan, seed, frac_bw=0.2, alpha=-0.7, rm_peak=2.0, snr=30.0):
    """Channel `chan` of a multi-frequency observation (the generators of `inputs`: one track set
    scaled per channel, power-law spectrum, Faraday rotation), with clean visibilities from the
    oracle's phi, one l2 block and the chi^2 radius."""
    stations = 8
    pairs = stations * (stations - 1) // 2
    wl = inputs.Workload("channels", n, M, stations, M // pairs + 2, levels, 1, 0, 0, snr, 0, seed)
    ratios = inputs.channel_ratios(nchan, frac_bw)
    uv0 = inputs.uv_coverage(wl, omega_max=inputs.EHT_OMEGA_MAX / float(ratios.max()))
    ratio = float(ratios[chan])
    uv = inputs.channel_uv(uv0, ratio)
    truth = inputs.channel_stokes(inputs.stokes_source(n, seed), ratio, alpha,
                                  inputs.rotation_measure_map(n, seed, rm_peak))
    w = np.ones(M, np.float32)
    clean = meas.phi(truth, uv, w.astype(np.float64))
    sigma = inputs.sigma_for_snr(clean, snr)
    Y = (clean + inputs.complex_noise(M, sigma, seed + 101 * chan)).astype(np.complex64)
    off = inputs.block_offsets(M, 1)
    eps = np.array([meas.chi2_epsilon(M, sigma)])
    prob = opd.Problem(n, levels, uv, w.astype(np.float64), Y.astype(np.complex128), off, eps)
    return {"uv": uv, "w": w, "Y": Y, "off": off, "eps": eps, "truth": truth, "sigma": sigma, "prob": prob}
