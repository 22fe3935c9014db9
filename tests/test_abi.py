"""The C-ABI library loads and exports every entry point include/polsara.h declares (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from oracle import wavelets as wav
from paper_1801_02417_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build_library()
    return binding.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "polsara.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("ps_create", "ps_set_measurements", "ps_set_sara_weights", "ps_pd_iterate", "ps_reweight",
                 "ps_get_stokes", "ps_get_state", "ps_set_state", "ps_destroy", "ps_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(binding.exported_symbols())


def test_library_filters_match_daubechies_definition(lib):
    """The library's host-side filter construction (long double, Durand-Kerner) agrees with the oracle's."""
    f = binding.ps_wavelet_filters()
    for p in range(1, 9):
        assert np.allclose(f[p - 1, :2 * p], wav.FILTERS[p], atol=1e-13)
        assert np.all(f[p - 1, 2 * p:] == 0)


def test_estimate_bytes_and_invalid_sizes(lib):
    assert binding.ps_estimate_bytes(1024, 6, 2_000_000) > 0
    assert binding.ps_estimate_bytes(100, 2, 10) == 0      # not a power of two
    assert binding.ps_estimate_bytes(64, 7, 10) == 0       # 2^7 does not divide 64


def test_create_rejects_bad_config_without_touching_a_device(lib):
    cfg = binding.ps_config(n=100, levels=2, mode=0, literal_ball=0, kernel_width=7, stop_maps=0,
                            tau=0, rho1=0, rho2=0, rho3=0)
    with pytest.raises(binding.PolsaraError) as e:
        binding.ps_create(cfg)
    assert e.value.status == binding.PS_EINVAL
    cfg.n, cfg.levels, cfg.kernel_width = 64, 2, 6
    with pytest.raises(binding.PolsaraError) as e:
        binding.ps_create(cfg)
    assert e.value.status == binding.PS_EINVAL


def test_create_validates_the_problem_and_stopping_fields_without_a_device(lib):
    """The ps_config fields of the problem statement and of the stopping rule (Section 5.5) are
    checked before any device call: oversampling other than 2, a negative gamma, sigma or
    tolerance, and a map count of the relative-change rule other than 3 or 4 are refused."""
    for field, bad in (("alpha", 3.0), ("gamma", -1.0), ("noise_sigma", -0.5), ("rel_tol", -1e-5),
                       ("resid_tol", float("nan")), ("np_tol", -0.5), ("zeta_sigma", float("inf")),
                       ("stop_maps", 2)):
        cfg = binding.ps_config(n=64, levels=2, mode=0, kernel_width=7)
        setattr(cfg, field, bad)
        with pytest.raises(binding.PolsaraError) as e:
            binding.ps_create(cfg)
        assert e.value.status == binding.PS_EINVAL, field
        assert "ps_create" in binding.ps_last_error(None)
