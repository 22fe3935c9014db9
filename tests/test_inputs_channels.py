"""Multi-frequency channel sets (per-channel Stokes maps and uv): pinned to the
physics they encode, on CPU. The source model: I and V follow ratio^alpha, the linear
polarization P = Q + iU follows the same power law and turns by 2 RM (lambda_c^2 -
lambda_0^2) (Faraday rotation); baselines in wavelengths scale with frequency."""
import math

import numpy as np
import pytest

from paper_1801_02417_gb300 import inputs


def test_channel_ratios_span_the_band():
    r = inputs.channel_ratios(8, 0.2)
    assert r.shape == (8,)
    assert math.isclose(r.min(), 0.9) and math.isclose(r.max(), 1.1)
    assert np.allclose(np.diff(r), 0.2 / 7)
    assert math.isclose(r.mean(), 1.0)
    assert np.array_equal(inputs.channel_ratios(1, 0.2), [1.0])


@pytest.mark.parametrize("ratio", [0.9, 1.0, 1.07])
def test_channel_stokes_power_law_and_faraday_rotation(ratio):
    n, alpha = 24, -0.7
    S0 = inputs.stokes_source(n, 5)
    rm = inputs.rotation_measure_map(n, 5, 2.0)
    Sc = inputs.channel_stokes(S0, ratio, alpha, rm)
    amp = ratio ** alpha
    assert np.allclose(Sc[0], amp * S0[0]) and np.allclose(Sc[3], amp * S0[3])
    P0 = S0[1] + 1j * S0[2]
    Pc = Sc[1] + 1j * Sc[2]
    assert np.allclose(np.abs(Pc), amp * np.abs(P0))
    # lambda^2 = lambda_0^2 / ratio^2, so the turn is 2 RM lambda_0^2 (ratio^-2 - 1).
    want = np.exp(2j * rm * (1.0 / ratio ** 2 - 1.0))
    mask = np.abs(P0) > 1e-9 * np.abs(P0).max()
    assert np.allclose(Pc[mask] / P0[mask], amp * want[mask])
    if ratio == 1.0:
        assert np.array_equal(Sc, S0)


def test_channels_keep_the_polarization_constraint():
    n = 32
    S0 = inputs.stokes_source(n, 9, 4)
    assert np.all(np.sqrt(S0[1] ** 2 + S0[2] ** 2 + S0[3] ** 2) <= S0[0] + 1e-12)
    rm = inputs.rotation_measure_map(n, 9, 3.0)
    for ratio in inputs.channel_ratios(5, 0.3):
        Sc = inputs.channel_stokes(S0, ratio, -0.7, rm)
        assert np.all(np.sqrt(Sc[1] ** 2 + Sc[2] ** 2 + Sc[3] ** 2) <= Sc[0] * (1 + 1e-12) + 1e-15)


def test_rotation_measure_map_is_bounded_and_signed():
    rm = inputs.rotation_measure_map(40, 2, 1.5)
    assert math.isclose(float(np.abs(rm).max()), 1.5)
    assert rm.min() < 0 < rm.max()


def test_channel_uv_scales_baselines():
    wl = inputs.WORKLOADS["img64_m2k"]
    ratios = inputs.channel_ratios(4, 0.2)
    uv0 = inputs.uv_coverage(wl, omega_max=inputs.EHT_OMEGA_MAX / ratios.max())
    for r in ratios:
        uv = inputs.channel_uv(uv0, r)
        assert np.allclose(uv, r * uv0)
        assert np.sqrt((uv ** 2).sum(1)).max() <= inputs.EHT_OMEGA_MAX * (1 + 1e-12) < math.pi
