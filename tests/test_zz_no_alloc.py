"""The allocation-free synthesis entry point (ps_apply_psi_static).

Some callers cannot call cudaMalloc: their device memory is all owned by another
allocator (a framework's caching allocator, a fixed pre-reserved pool), or they
must not risk an allocation failing or stalling in the middle of a run. For them
ps_apply_psi_static computes S = Psi A with its level scratch in a static device
array, allocating nothing. This file checks it through the C ABI against the
ordinary handle-based ps_apply_psi on two calls in a row (the second call reuses
the scratch the first one left behind), and that oversize requests are refused.
It is collected last so that a stop-at-first-failure run has already run every
other test.
"""
import numpy as np
import pytest

from paper_1801_02417_gb300 import _build
from paper_1801_02417_gb300 import binding as B

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the SARA operator tolerance of the parity tests


@pytest.fixture(scope="module")
def lib():
    _build.build_library()
    return B.lib()


def test_static_scratch_synthesis_matches_handle_path(lib):
    import torch
    n, levels = 128, 4          # levels 128, 64, 32 take the tiled kernels, 16 the small-level kernel
    cfg = B.ps_config(n=n, levels=levels, mode=0, literal_ball=0, kernel_width=7, reserved=0,
                      tau=0, rho1=0, rho2=0, rho3=0)
    h = B.ps_create(cfg)
    try:
        for call in range(2):
            A = np.random.default_rng(100 + call).normal(size=(4, 9, n, n)).astype(np.float32)
            expect = np.empty((4, n, n), np.float32)
            B.ps_apply_psi(h, A, expect)
            Ad = torch.from_numpy(A).cuda()
            Sd = torch.full((4, n, n), float("nan"), device="cuda")
            B.ps_apply_psi_static(Ad, Sd, n, levels, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = Sd.cpu().numpy()
            assert np.all(np.isfinite(got))
            rel = np.linalg.norm(got - expect) / np.linalg.norm(expect)
            assert rel <= TOL, (call, rel)
    finally:
        B.ps_destroy(h)


def test_static_scratch_rejects_sizes_beyond_its_limit(lib):
    import torch
    A = torch.zeros(16, device="cuda")
    S = torch.zeros(16, device="cuda")
    with pytest.raises(B.PolsaraError) as e:
        B.ps_apply_psi_static(A, S, 512, 4)
    assert e.value.status == B.PS_EINVAL
    assert "static scratch" in B.ps_last_error(None)
