"""Parity at the benchmark's full size: 1024 x 1024 4-Stokes, 2,000,000 rows, 32 blocks, 6 levels.

The oracle cannot run whole iterations at this size (its direct DFT costs
~8e12 complex MACs per phi), so outputs are compared where the oracle can
compute them one by one: phi on sampled rows, phi^dagger on sampled pixels, the
SARA transforms on whole maps, and the per-pixel primal/epigraph step of one
iteration at sampled pixels. Same tolerances as the small-size parity tests.
"""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import primal_dual as opd
from oracle import prox
from oracle import wavelets as wav
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300 import inputs
from paper_1801_02417_gb300.solver import PolarizedSARA

pytestmark = pytest.mark.gpu

WL = inputs.WORKLOADS["img1024_m2m"]


@pytest.fixture(scope="module")
def big():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    uv = inputs.uv_coverage(WL)
    w = inputs.visibility_weights(WL.M, WL.seed, 0.2).astype(np.float32)
    truth = inputs.stokes_source(WL.n, WL.seed, WL.n_compact).astype(np.float32)
    rng = np.random.default_rng(5)
    Y = (rng.normal(size=(WL.M, 4)) + 1j * rng.normal(size=(WL.M, 4))).astype(np.complex64)
    off = inputs.block_offsets(WL.M, WL.nblocks)
    eps = np.full(WL.nblocks, 1e3)
    s = PolarizedSARA(WL.n, WL.levels)
    s.set_measurements(uv, Y, w, off, eps)
    yield {"s": s, "uv": uv, "w": w, "truth": truth, "Y": Y, "off": off, "eps": eps, "rng": rng}
    s.close()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_phi_on_sampled_rows(big):
    s, uv, w = big["s"], big["uv"], big["w"]
    out = np.empty((WL.M, 4), np.complex64)
    B.ps_apply_phi(s.h, big["truth"], out)
    rows = np.sort(big["rng"].choice(WL.M, size=96, replace=False))
    ref = meas.phi(big["truth"].astype(np.float64), uv[rows], w[rows].astype(np.float64))
    assert _rel(out[rows], ref) <= 1e-5


def test_phi_adjoint_on_sampled_pixels(big):
    s, uv, w, Y = big["s"], big["uv"], big["w"], big["Y"]
    img = np.empty((4, WL.n, WL.n), np.float32)
    B.ps_apply_phi_adjoint(s.h, Y, img)
    pix = np.stack([big["rng"].integers(0, WL.n, 12), big["rng"].integers(0, WL.n, 12)], axis=1)
    pix = np.concatenate([pix, [[0, 0], [WL.n - 1, WL.n - 1], [WL.n // 2, WL.n // 2]]])
    ref = meas.phi_adjoint_at(Y.astype(np.complex128), uv, w.astype(np.float64), WL.n, pix)
    got = img[:, pix[:, 0], pix[:, 1]]
    assert _rel(got, ref) <= 1e-5


def test_phi_every_degridding_choice(big):
    """Every degridding launch choice at full size on sampled rows; the whole outputs of
    all choices agree within FP32 rounding."""
    s, uv, w = big["s"], big["uv"], big["w"]
    rows = np.sort(big["rng"].choice(WL.M, size=64, replace=False))
    ref = meas.phi(big["truth"].astype(np.float64), uv[rows], w[rows].astype(np.float64))
    saved = B.ps_get_tuning(s.h)
    outs = []
    try:
        for choice in range(3):
            B.ps_set_tuning(s.h, saved[:1] + [choice] + saved[2:])
            out = np.empty((WL.M, 4), np.complex64)
            B.ps_apply_phi(s.h, big["truth"], out)
            assert _rel(out[rows], ref) <= 1e-5, choice
            outs.append(out)
    finally:
        B.ps_set_tuning(s.h, saved)
    for choice, out in enumerate(outs[1:], 1):
        assert _rel(out, outs[0]) <= 1e-6, choice


def test_phi_adjoint_every_gridding_choice(big):
    """Every gridding launch choice at full size on sampled pixels; the whole maps of all
    choices agree within the FP32 tolerance of the atomics' order."""
    s, uv, w, Y = big["s"], big["uv"], big["w"], big["Y"]
    pix = np.stack([big["rng"].integers(0, WL.n, 10), big["rng"].integers(0, WL.n, 10)], axis=1)
    ref = meas.phi_adjoint_at(Y.astype(np.complex128), uv, w.astype(np.float64), WL.n, pix)
    saved = B.ps_get_tuning(s.h)
    maps = []
    try:
        for choice in range(5):
            B.ps_set_tuning(s.h, saved[:2] + [choice] + saved[3:])
            img = np.empty((4, WL.n, WL.n), np.float32)
            B.ps_apply_phi_adjoint(s.h, Y, img)
            assert _rel(img[:, pix[:, 0], pix[:, 1]], ref) <= 1e-5, choice
            maps.append(img)
    finally:
        B.ps_set_tuning(s.h, saved)
    for choice, img in enumerate(maps[1:], 1):
        assert _rel(img, maps[0]) <= 1e-6, choice


def test_sara_transforms_full_maps(big):
    s = big["s"]
    S = big["truth"]
    A = np.empty((4, 9, WL.n, WL.n), np.float32)
    B.ps_apply_psi_adjoint(s.h, S, A)
    ref = wav.psi_adjoint(S[:1].astype(np.float64), WL.levels)[0]
    assert _rel(A[0], ref) <= 1e-6
    back = np.empty((4, WL.n, WL.n), np.float32)
    B.ps_apply_psi(s.h, A, back)
    ref_back = wav.psi(A[2:3].astype(np.float64), WL.levels)[0]
    assert _rel(back[2], ref_back) <= 1e-6


def test_one_iteration_per_pixel_step_at_sampled_pixels(big):
    """S', Z', C', D' of one iteration at sampled pixels, from the oracle's Psi A and phi^dagger B there."""
    s, uv, w = big["s"], big["uv"], big["w"]
    n, M = WL.n, WL.M
    rng = np.random.default_rng(11)
    st = {"S": (0.1 * rng.normal(size=(4, n, n))).astype(np.float32),
          "Z": (0.1 * rng.normal(size=(2, n, n))).astype(np.float32),
          "A": (0.01 * rng.normal(size=(4, 9, n, n))).astype(np.float32),
          "B": (1e-3 * (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4)))).astype(np.complex64),
          "C": (0.1 * rng.normal(size=(4, n, n))).astype(np.float32),
          "D": (0.1 * rng.normal(size=(2, n, n))).astype(np.float32)}
    s.set_sara_weights(None, 0.05)
    s.set_state(st)
    s.set_mode(B.PS_POLARIZED)
    par = s.params()
    s.pd_iterate(1)
    got = s.get_state()
    pix = np.stack([rng.integers(0, n, 10), rng.integers(0, n, 10)], axis=1)
    # Oracle pieces at those pixels: Psi A (whole maps, then sampled) and phi^dagger B.
    PsiA = wav.psi(st["A"].astype(np.float64), WL.levels)[:, pix[:, 0], pix[:, 1]]
    AdjB = meas.phi_adjoint_at(st["B"].astype(np.complex128), uv, w.astype(np.float64), n, pix)
    S0 = st["S"][:, pix[:, 0], pix[:, 1]].astype(np.float64)
    C0 = st["C"][:, pix[:, 0], pix[:, 1]].astype(np.float64)
    Z0 = st["Z"][:, pix[:, 0], pix[:, 1]].astype(np.float64)
    D0 = st["D"][:, pix[:, 0], pix[:, 1]].astype(np.float64)
    tau, r3 = par["tau"], par["rho3"]
    S1 = prox.proj_U(S0 - tau * (PsiA + AdjB + C0))
    Z1 = prox.proj_V(Z0 - tau * D0)
    Sb, Zb = 2 * S1 - S0, 2 * Z1 - Z0
    Ct, Dt = C0 + r3 * Sb, D0 + r3 * Zb
    c1, d1 = prox.proj_E1(Ct[0] / r3, Dt[0] / r3)
    R2, d2 = prox.proj_E2(Ct[1:4] / r3, Dt[1] / r3)
    C1 = np.concatenate([(Ct[0] - r3 * c1)[None], Ct[1:4] - r3 * R2])
    D1 = np.stack([Dt[0] - r3 * d1, Dt[1] - r3 * d2])
    assert _rel(got["S"][:, pix[:, 0], pix[:, 1]], S1) <= 2e-5
    assert _rel(got["Z"][:, pix[:, 0], pix[:, 1]], Z1) <= 2e-5
    assert _rel(got["C"][:, pix[:, 0], pix[:, 1]], C1) <= 2e-5
    assert _rel(got["D"][:, pix[:, 0], pix[:, 1]], D1) <= 2e-5


def test_sara_every_launch_choice_full_maps(big):
    """Every finest-level synthesis form (the persistent one loops over several (tile, map)
    units per CTA only at this size) and every level-1 analysis form against the oracle's
    transforms of one map, and all forms agree with each other over the four maps."""
    s = big["s"]
    rng = np.random.default_rng(17)
    A = rng.normal(size=(4, 9, WL.n, WL.n)).astype(np.float32)
    S = big["truth"]
    ref_syn = wav.psi(A[1:2].astype(np.float64), WL.levels)[0]
    ref_ana = wav.psi_adjoint(S[3:4].astype(np.float64), WL.levels)[0]
    saved = B.ps_get_tuning(s.h)
    outs, coefs = [], []
    try:
        for syn in range(3):
            B.ps_set_tuning(s.h, [syn] + saved[1:])
            back = np.empty((4, WL.n, WL.n), np.float32)
            B.ps_apply_psi(s.h, A, back)
            assert _rel(back[1], ref_syn) <= 1e-6, syn
            outs.append(back)
        for ana in range(6):
            B.ps_set_tuning(s.h, saved[:3] + [ana])
            C = np.empty((4, 9, WL.n, WL.n), np.float32)
            B.ps_apply_psi_adjoint(s.h, S, C)
            assert _rel(C[3], ref_ana) <= 1e-6, ana
            coefs.append(C)
    finally:
        B.ps_set_tuning(s.h, saved)
    for o in outs[1:]:
        assert _rel(o, outs[0]) <= 1e-6
    for c in coefs[1:]:
        assert _rel(c, coefs[0]) <= 1e-6


# Rows and columns on the image edges, the centre and the boundaries of the 32- and 64-wide
# SARA tiles and of the FFT halves, plus seeded interior ones.
_EDGE_LINES = [0, 1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 255, 256, 257, 511, 512, 513, 767, 768, 1021, 1022, 1023]


def test_phi_adjoint_on_boundary_grid_with_elementwise_bound(big):
    """phi^dagger of the 2M rows on the 1,600 pixels where 40 rows cross 40 columns chosen on tile,
    centre and edge boundaries (and at random): relative l2 within 1e-5 and every element within
    1e-5 of the largest value, so no boundary error hides in a global norm."""
    s, uv, w, Y = big["s"], big["uv"], big["w"], big["Y"]
    img = np.empty((4, WL.n, WL.n), np.float32)
    B.ps_apply_phi_adjoint(s.h, Y, img)
    rng = np.random.default_rng(19)
    lines = sorted(set(_EDGE_LINES) | set(rng.integers(0, WL.n, 18).tolist()))
    ys, xs = lines[:40], lines[-40:]
    ref = meas.phi_adjoint_grid(Y.astype(np.complex128), uv, w.astype(np.float64), WL.n, ys, xs)
    got = img[:, ys][:, :, xs].astype(np.float64)
    assert _rel(got, ref) <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_one_iteration_duals_at_full_size():
    """One iteration at 1024^2 / 2M rows from a random state: the l1 dual A (every coefficient,
    steps 5-6: clamp(A + rho1 Psi^dagger X^bar, +-gamma W) with the oracle's Psi^dagger of the
    GPU's X^bar = 2 S' - S) and the data dual B of one block made of 256 rows (steps 7-8: the
    oracle's direct DFT of X^bar on those rows, the block's ball factor, B = c_b (B~/rho2 - Y)),
    within the one-iteration bound 2e-5."""
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    n, M = WL.n, WL.M
    uv = inputs.uv_coverage(WL)
    w = inputs.visibility_weights(M, WL.seed, 0.2).astype(np.float32)
    rng = np.random.default_rng(23)
    Y = (0.05 * (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4)))).astype(np.complex64)
    off = np.concatenate([[0, 256], inputs.block_offsets(M - 256, 31)[1:] + 256]).astype(np.int64)
    eps = np.full(32, 30.0)
    eps[0] = 0.5
    st = {"S": (0.1 * rng.normal(size=(4, n, n))).astype(np.float32),
          "Z": (0.1 * rng.normal(size=(2, n, n))).astype(np.float32),
          "A": (0.01 * rng.normal(size=(4, 9, n, n))).astype(np.float32),
          "C": (0.1 * rng.normal(size=(4, n, n))).astype(np.float32),
          "D": (0.1 * rng.normal(size=(2, n, n))).astype(np.float32)}
    W = rng.uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.01
    with PolarizedSARA(n, WL.levels) as s:
        s.set_measurements(uv, Y, w, off, eps)
        par = s.params()
        # B on the scale of rho2 phi(X^bar) (per row ~ 0.1 sqrt(N) = 100), so that both terms of
        # B~ = B + rho2 phi(X^bar) count in the comparison.
        st["B"] = (par["rho2"] * 50.0 * (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4)))).astype(np.complex64)
        s.set_sara_weights(W, gamma)
        s.set_state(st)
        s.pd_iterate(1)
        got = s.get_state()
    Xb = 2.0 * got["S"].astype(np.float64) - st["S"].astype(np.float64)
    T = gamma * W.astype(np.float64)
    A_ref = np.clip(st["A"] + par["rho1"] * wav.psi_adjoint(Xb, WL.levels), -T, T)
    assert _rel(got["A"], A_ref) <= 2e-5
    rows = np.arange(256)
    w64 = w.astype(np.float64)
    Bt = st["B"][rows].astype(np.complex128) + par["rho2"] * meas.phi(Xb, uv[rows], w64[rows])
    R = Bt / par["rho2"] - Y[rows].astype(np.complex128)
    r = np.linalg.norm(R)
    c_b = par["rho2"] * (1.0 - min(1.0, eps[0] / r))
    assert c_b > 0                                   # the ball constraint is active for this block
    assert _rel(got["B"][rows], c_b * R) <= 2e-5
