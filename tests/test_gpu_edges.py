"""GPU parity at the edges of the problem statement: no measurements at all, more l2 blocks
than the degridding kernel's per-warp bins (its shared-atomic path) and blocks of a single
row, data that are exactly zero, the largest image the ABI accepts (2048^2), and a single
wavelet level. Same bounds as the other parity tests: operators within 1e-5 (1e-6 for the
SARA transforms), k iterations from a random state within 2e-5 k of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import primal_dual as opd
from oracle import wavelets as wav
from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300 import inputs
from paper_1801_02417_gb300.solver import PolarizedSARA
from problems import make_problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1801_02417_gb300 import _build
    _build.build_library()
    B.lib()


def _random_state(n, M, seed, scale=0.05):
    st = inputs.random_state(n, M, seed, scale)
    return {k: (v.astype(np.complex64) if k == "B" else v.astype(np.float32)) for k, v in st.items()}


def _iterate_against_oracle(s, prob, st32, T, p, iters, keys):
    ref = {k: v.astype(np.complex128 if k == "B" else np.float64) for k, v in st32.items()}
    s.set_state(st32)
    s.pd_iterate(iters)
    for _ in range(iters):
        ref = opd.pd_iteration(ref, prob, T, p, opd.POLARIZED)
    got = s.get_state()
    for k in keys:
        err = rel_err(got[k], ref[k])
        assert err <= 2e-5 * iters, (k, err)


def test_no_measurements_iterates_like_oracle():
    """M = 0: the data term is absent (phi has no rows, ||phi||^2 = 0), so the library takes
    rho2 = 1 and tau = 0.99 / (rho1 + rho3); Algorithm 1 reduces to the sparsity and
    polarization terms, and three iterations match the oracle's on the same empty problem."""
    n, levels = 32, 3
    uv = np.zeros((0, 2))
    Y = np.zeros((0, 4), np.complex64)
    w = np.zeros(0, np.float32)
    off = np.zeros(1, np.int64)
    eps = np.zeros(0)
    prob = opd.Problem(n, levels, uv, w.astype(np.float64), Y.astype(np.complex128), off, eps)
    p = opd.step_sizes(0.0, opd.POLARIZED, rho2=1.0)
    W = np.random.default_rng(40).uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.02
    with PolarizedSARA(n, levels) as s:
        s.set_measurements(uv, Y, w, off, eps)
        par = s.params()
        assert par["opnorm_sq"] == 0.0
        assert abs(par["rho2"] - 1.0) < 1e-15 and abs(par["tau"] - p.tau) < 1e-12
        s.set_sara_weights(W, gamma)
        _iterate_against_oracle(s, prob, _random_state(n, 0, 41), gamma * W.astype(np.float64), p, 3,
                                ("S", "Z", "A", "C", "D"))


@pytest.mark.parametrize("M,nblocks", [(1500, 100), (300, 300)])
def test_many_and_single_row_blocks_iterate_like_oracle(M, nblocks):
    """100 blocks (beyond the 64 per-warp FP64 bins of the degridding kernel: shared atomic
    bins) and 300 blocks of one row each (every row its own l2 ball): per-block radii and
    ball factors through three iterations against the oracle."""
    n, levels = 32, 3
    pb = make_problem(n, M, levels, nblocks, seed=42)
    prob = pb["prob"]
    p = opd.step_sizes(meas.op_norm_sq_lanczos(pb["uv"], prob.w, n), opd.POLARIZED)
    W = np.random.default_rng(43).uniform(0.2, 1.0, size=(4, 9, n, n)).astype(np.float32)
    gamma = 0.02
    with PolarizedSARA(n, levels, tau=p.tau, rho1=p.rho1, rho2=p.rho2, rho3=p.rho3) as s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        s.set_sara_weights(W, gamma)
        _iterate_against_oracle(s, prob, _random_state(n, M, 44), gamma * W.astype(np.float64), p, 3,
                                ("S", "Z", "A", "B", "C", "D"))


def test_zero_data_keep_the_zero_state():
    """Y = 0 from the zero state is a fixed point of Algorithm 1 (every step maps zeros to
    zeros; the ball factor of a block whose residual is exactly zero is 0, not 0/0): the
    state stays exactly zero and finite."""
    n, levels, M = 32, 3, 800
    pb = make_problem(n, M, levels, 2, seed=45)
    zeros = np.zeros((M, 4), np.complex64)
    with PolarizedSARA(n, levels) as s:
        s.set_measurements(pb["uv"], zeros, pb["w"], pb["off"], pb["eps"])
        s.set_sara_weights(None, 0.02)
        s.pd_iterate(5)
        st = s.get_state()
    for k, v in st.items():
        assert np.all(v == 0), k


def test_largest_image_operators():
    """n = 2048 (the largest side the ABI accepts), 5 levels, 100,000 rows: the SARA pair is a
    tight frame (Psi Psi^dagger = Id) and adjoint to FP32 rounding; phi on sampled rows and
    phi^dagger on sampled pixels (tile and window edges among them) against the oracle's
    direct sums."""
    n, levels, M = 2048, 5, 100_000
    wl = inputs.Workload("edge2048", n, M, 10, M // 45 + 2, levels, 4, 0, 0, 30.0, 0, 46)
    uv = inputs.uv_coverage(wl)
    w = inputs.visibility_weights(M, 46, 0.2).astype(np.float32)
    rng = np.random.default_rng(47)
    Y = (rng.normal(size=(M, 4)) + 1j * rng.normal(size=(M, 4))).astype(np.complex64)
    off = inputs.block_offsets(M, 4)
    X = inputs.stokes_source(n, 46).astype(np.float32)
    with PolarizedSARA(n, levels) as s:
        s.set_measurements(uv, Y, w, off, np.full(4, 1e3))
        A = np.empty((4, 9, n, n), np.float32)
        B.ps_apply_psi_adjoint(s.h, X, A)
        back = np.empty((4, n, n), np.float32)
        B.ps_apply_psi(s.h, A, back)
        assert rel_err(back, X) <= 1e-6
        R = rng.normal(size=(4, 9, n, n)).astype(np.float32)
        PR = np.empty((4, n, n), np.float32)
        B.ps_apply_psi(s.h, R, PR)
        lhs = float(np.dot(A.astype(np.float64).ravel(), R.astype(np.float64).ravel()))
        rhs = float(np.dot(X.astype(np.float64).ravel(), PR.astype(np.float64).ravel()))
        assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(A) * np.linalg.norm(R)
        del A, R, PR
        out = np.empty((M, 4), np.complex64)
        B.ps_apply_phi(s.h, X, out)
        rows = np.sort(rng.choice(M, size=32, replace=False))
        ref = meas.phi(X.astype(np.float64), uv[rows], w[rows].astype(np.float64))
        assert rel_err(out[rows], ref) <= 1e-5
        img = np.empty((4, n, n), np.float32)
        B.ps_apply_phi_adjoint(s.h, Y, img)
    pix = np.array([[0, 0], [n - 1, n - 1], [n // 2, n // 2], [15, 16], [16, 15], [1023, 1024], [2047, 0],
                    [0, 2047], [777, 1301], [1500, 64]])
    ref = meas.phi_adjoint_at(Y.astype(np.complex128), uv, w.astype(np.float64), n, pix)
    assert rel_err(img[:, pix[:, 0], pix[:, 1]], ref) <= 1e-5


@pytest.mark.parametrize("n", [64, 256])
def test_single_level_transforms_match_oracle(n):
    """One wavelet level (the coarsest approximation is half the image): Psi and Psi^dagger
    against the oracle."""
    pb = make_problem(n, 64, 1, 1, seed=48)
    rng = np.random.default_rng(49)
    S = rng.normal(size=(4, n, n)).astype(np.float32)
    A = rng.normal(size=(4, 9, n, n)).astype(np.float32)
    with PolarizedSARA(n, 1) as s:
        s.set_measurements(pb["uv"], pb["Y"], pb["w"], pb["off"], pb["eps"])
        Ag = np.empty((4, 9, n, n), np.float32)
        B.ps_apply_psi_adjoint(s.h, S, Ag)
        Sg = np.empty((4, n, n), np.float32)
        B.ps_apply_psi(s.h, A, Sg)
    assert rel_err(Ag, wav.psi_adjoint(S.astype(np.float64), 1)) <= 1e-6
    assert rel_err(Sg, wav.psi(A.astype(np.float64), 1)) <= 1e-6
