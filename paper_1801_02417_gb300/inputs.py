"""Seeded synthetic inputs for full-polarization (I, Q, U, V) imaging problems.

This module draws random quantities only: truth Stokes maps, Earth-rotation uv
tracks, visibility weights, noise realisations and block partitions. It holds
none of the imaging method's arithmetic (no measurement operator, no wavelet,
no projection), so both the FP64 oracle and the CUDA path can take their inputs
from it. Clean visibilities are formed by whichever operator the caller uses;
the noise matrix E of the data model Y = phi(S) + E (Section 2.1, Eq. RIME_disc)
is drawn here and passed in.

The workloads follow the paper's simulation setup (Section 5.1): an EHT-like
VLBI array whose longest baseline maps to 0.44 rad/pixel (7.2 Glambda at 2 uas
pixels), compact sources in which Q and U are much fainter than I, V near zero,
and i.i.d. complex Gaussian noise of variance sigma^2 (sigma^2/2 per real part).
The paper's own datasets (EHT coverage file, M87 model images) are not
available, so these seeded stand-ins take their shapes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Longest projected baseline of the paper's EHT coverage (7.2 Glambda) times
# the 2 micro-arcsecond pixel (9.696e-12 rad), in radians per pixel.
EHT_OMEGA_MAX = 2.0 * math.pi * 7.2e9 * (2e-6 / 3600.0 * math.pi / 180.0)
EARTH_RADIUS_M = 6.371e6
BASE_SEED = 20180108


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic imaging problem: image side, visibility count and solver budget."""
    name: str
    n: int                 # image side (N = n*n pixels per Stokes map)
    M: int                 # visibilities (rows of Y, 4 correlations each)
    stations: int
    dumps: int             # time samples over the 12 h track
    levels: int            # wavelet decomposition levels
    nblocks: int           # l2 data blocks
    iterations: int        # total primal-dual iterations
    reweights: int         # reweighting steps (Algorithm 2)
    snr_db: float          # input SNR of the noisy data
    n_compact: int = 0     # extra compact polarized components
    seed: int = BASE_SEED


WORKLOADS = {
    # 64x64, M=2000, 8 stations, one block, 4 levels, 300 iterations, 3 reweights.
    "img64_m2k": Workload("img64_m2k", 64, 2000, 8, 72, 4, 1, 300, 3, 30.0, 0, BASE_SEED + 0),
    # 256x256, M=50k, 10 stations, 8 blocks, 500 iterations, 5 reweights.
    "img256_m50k": Workload("img256_m50k", 256, 50000, 10, 1112, 4, 8, 500, 5, 30.0, 0, BASE_SEED + 1),
    # 1024x1024, M=2M, 64 stations, 32 blocks, 6 levels, 1000 iterations,
    # plus 200 random compact polarized components.
    "img1024_m2m": Workload("img1024_m2m", 1024, 2000000, 64, 993, 6, 32, 1000, 0, 30.0, 200, BASE_SEED + 2),
}


def _smooth_field(rng: np.random.Generator, n: int, n_modes: int = 6, kmax: float = 3.0) -> np.ndarray:
    """A smooth random field on [0,1]: a sum of a few low-frequency cosines, rescaled."""
    p = np.arange(n)[:, None] / n
    q = np.arange(n)[None, :] / n
    f = np.zeros((n, n))
    for _ in range(n_modes):
        kx, ky = rng.uniform(-kmax, kmax, size=2)
        ph = rng.uniform(0, 2 * math.pi)
        f += rng.uniform(0.5, 1.0) * np.cos(2 * math.pi * (kx * q + ky * p) + ph)
    f -= f.min()
    mx = f.max()
    return f / mx if mx > 0 else f


def stokes_source(n: int, seed: int, n_compact: int = 0) -> np.ndarray:
    """Truth Stokes maps, shape (4, n, n) in the order I, Q, U, V (float64).

    I: three Gaussians (sigma 2-6 px at n=64, scaled by n/64) plus a ring of
    radius 12 px (scaled by n/64) with a 1.5 px Gaussian cross-section.
    Q = m I cos(2 chi), U = m I sin(2 chi) with m a smooth field in [0, 0.6] and
    chi a smooth EVPA field; V = 0.01 I. Every pixel then satisfies
    sqrt(Q^2+U^2+V^2) <= I. ``n_compact`` adds that many compact (sigma 1-2 px)
    Gaussians, each with its own fractional polarization and EVPA.
    """
    rng = np.random.default_rng(seed)
    s = n / 64.0
    p = np.arange(n)[:, None] - n / 2
    q = np.arange(n)[None, :] - n / 2
    I = np.zeros((n, n))
    for _ in range(3):
        cy, cx = rng.uniform(-0.25 * n, 0.25 * n, size=2)
        sig = rng.uniform(2.0, 6.0) * s
        amp = rng.uniform(0.3, 1.0)
        I += amp * np.exp(-((q - cx) ** 2 + (p - cy) ** 2) / (2 * sig * sig))
    r = np.sqrt(p.astype(float) ** 2 + q.astype(float) ** 2)
    I += 0.5 * np.exp(-((r - 12.0 * s) ** 2) / (2 * 1.5 ** 2))
    m = 0.6 * _smooth_field(rng, n)
    chi = math.pi * _smooth_field(rng, n)
    Q = m * I * np.cos(2 * chi)
    U = m * I * np.sin(2 * chi)
    for _ in range(n_compact):
        cy, cx = rng.uniform(-0.45 * n, 0.45 * n, size=2)
        sig = rng.uniform(1.0, 2.0)
        amp = rng.uniform(0.05, 0.5)
        mc = rng.uniform(0.0, 0.6)
        chic = rng.uniform(0.0, math.pi)
        g = amp * np.exp(-((q - cx) ** 2 + (p - cy) ** 2) / (2 * sig * sig))
        I += g
        Q += mc * g * math.cos(2 * chic)
        U += mc * g * math.sin(2 * chic)
    V = 0.01 * I
    return np.stack([I, Q, U, V])


def station_positions(n_stations: int, rng: np.random.Generator) -> np.ndarray:
    """Seeded random ECEF station positions on an Earth-radius sphere, shape (n, 3), metres."""
    v = rng.normal(size=(n_stations, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return EARTH_RADIUS_M * v


def earth_rotation_uv(n_stations: int, n_dumps: int, seed: int, dec_deg: float = 12.0,
                      hours: float = 12.0) -> np.ndarray:
    """uv tracks (metres) of every station pair over ``hours`` of Earth rotation.

    Textbook projection of a baseline (Bx, By, Bz) towards a source at hour angle
    H and declination dec: u = sin H Bx + cos H By,
    v = -sin(dec) cos H Bx + sin(dec) sin H By + cos(dec) Bz.
    Returns shape (n_dumps * n_pairs, 2), rows ordered by pair then time.
    """
    rng = np.random.default_rng(seed)
    pos = station_positions(n_stations, rng)
    a, b = np.triu_indices(n_stations, k=1)
    B = pos[b] - pos[a]                                    # (pairs, 3)
    H = np.linspace(-hours / 2, hours / 2, n_dumps) * (2 * math.pi / 24.0)
    dec = math.radians(dec_deg)
    sH, cH = np.sin(H)[None, :], np.cos(H)[None, :]
    Bx, By, Bz = B[:, 0:1], B[:, 1:2], B[:, 2:3]
    u = sH * Bx + cH * By
    v = -math.sin(dec) * cH * Bx + math.sin(dec) * sH * By + math.cos(dec) * Bz
    return np.stack([u.ravel(), v.ravel()], axis=1)


def uv_coverage(w: Workload, omega_max: float = EHT_OMEGA_MAX) -> np.ndarray:
    """Sampled frequencies in radians per pixel, shape (M, 2), float64.

    Tracks are scaled so the longest baseline sits at ``omega_max`` and a seeded
    subset of M rows is kept (in track order).
    """
    uv = earth_rotation_uv(w.stations, w.dumps, w.seed)
    if uv.shape[0] < w.M:
        raise ValueError(f"{w.name}: tracks give {uv.shape[0]} rows < M={w.M}")
    rng = np.random.default_rng(w.seed + 7)
    keep = np.sort(rng.choice(uv.shape[0], size=w.M, replace=False))
    uv = uv[keep]
    rmax = np.sqrt((uv ** 2).sum(1)).max()
    return uv * (omega_max / rmax)


# ---- multi-frequency (hyperspectral) channel sets: the polarization constraint acts
# at each wavelength on its own (Section 6), so each channel is an independent
# Stokes imaging problem; these generators give the channels' inputs.
def channel_ratios(nchan: int, frac_bw: float) -> np.ndarray:
    """Channel frequencies over the reference frequency, evenly over the band [1 - bw/2, 1 + bw/2]."""
    if nchan == 1:
        return np.ones(1)
    return 1.0 + frac_bw * (np.arange(nchan) / (nchan - 1) - 0.5)


def channel_uv(uv0: np.ndarray, ratio: float) -> np.ndarray:
    """Sampled frequencies of a channel: baselines in wavelengths grow with frequency."""
    return uv0 * ratio


def rotation_measure_map(n: int, seed: int, peak: float) -> np.ndarray:
    """Smooth Faraday depth map, expressed as RM lambda_0^2 in radians, |.| <= peak."""
    rng = np.random.default_rng(seed + 17)
    f = 2.0 * _smooth_field(rng, n) - 1.0
    return peak * f / max(float(np.abs(f).max()), 1e-30)


def channel_stokes(S0: np.ndarray, ratio: float, alpha: float, rm_l0sq: np.ndarray) -> np.ndarray:
    """Stokes maps of one channel from the reference-frequency maps S0 (4, n, n).

    I and V follow a power law ratio^alpha; the linear polarization P = Q + iU follows
    the same law and turns by 2 RM (lambda_c^2 - lambda_0^2) = 2 RM lambda_0^2 (ratio^-2 - 1)
    (Faraday rotation), which keeps |P| and so the constraint sqrt(Q^2+U^2+V^2) <= I.
    """
    amp = ratio ** alpha
    turn = 2.0 * rm_l0sq * (ratio ** -2 - 1.0)
    c, s = np.cos(turn), np.sin(turn)
    Q, U = S0[1], S0[2]
    return np.stack([amp * S0[0], amp * (c * Q - s * U), amp * (s * Q + c * U), amp * S0[3]])


def random_uv(M: int, seed: int, omega_max: float) -> np.ndarray:
    """Uniformly scattered frequencies in a square of half-width ``omega_max`` rad/pixel."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-omega_max, omega_max, size=(M, 2))


def visibility_weights(M: int, seed: int, spread: float = 0.0) -> np.ndarray:
    """Per-row weights: ones when ``spread`` is 0, else uniform in [1-spread, 1+spread]."""
    if spread == 0.0:
        return np.ones(M)
    rng = np.random.default_rng(seed + 11)
    return rng.uniform(1.0 - spread, 1.0 + spread, size=M)


def complex_noise(M: int, sigma: float, seed: int) -> np.ndarray:
    """i.i.d. complex Gaussian noise matrix E (M, 4): variance sigma^2/2 per real and imaginary part."""
    rng = np.random.default_rng(seed + 13)
    s = sigma / math.sqrt(2.0)
    return rng.normal(scale=s, size=(M, 4)) + 1j * rng.normal(scale=s, size=(M, 4))


def sigma_for_snr(clean_vis: np.ndarray, snr_db: float) -> float:
    """Noise level giving the requested input SNR: ||clean||^2 / E||E||^2 = 10^(snr/10)."""
    p = float(np.sum(np.abs(clean_vis) ** 2)) / clean_vis.size
    return math.sqrt(p * 10.0 ** (-snr_db / 10.0))


def block_offsets(M: int, nblocks: int) -> np.ndarray:
    """Contiguous, near-equal l2 data blocks: int64 offsets of length nblocks+1."""
    return np.round(np.linspace(0, M, nblocks + 1)).astype(np.int64)


def random_state(n: int, M: int, seed: int, scale: float = 1.0) -> dict:
    """Random primal/dual state arrays (float64/complex128) for one-step parity tests."""
    rng = np.random.default_rng(seed)
    N = n * n
    return {
        "S": scale * rng.normal(size=(4, n, n)),
        "Z": scale * rng.normal(size=(2, n, n)),
        "A": scale * rng.normal(size=(4, 9, n, n)),
        "B": scale * (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))),
        "C": scale * rng.normal(size=(4, n, n)),
        "D": scale * rng.normal(size=(2, n, n)),
    }
