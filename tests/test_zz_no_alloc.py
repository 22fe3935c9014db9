"""The allocation-free synthesis entry point (ps_apply_psi_static).

Some callers cannot call cudaMalloc: their device memory is all owned by another
allocator (a framework's caching allocator, a fixed pre-reserved pool), or they
must not risk an allocation failing or stalling in the middle of a run. For them
ps_apply_psi_static computes S = Psi A with its level scratch in a static device
array, allocating nothing. This file checks it through the C ABI against the
ordinary handle-based ps_apply_psi and against the oracle's wavelet synthesis on
two calls in a row (the second call reuses the scratch the first one left
behind), at the sizes that take every synthesis kernel up to the scratch's limit;
that a repeated call changes neither the device's free memory nor torch's
reserved memory; that a bounded wait that gives up is reported by ps_static_status;
and that oversize requests and host pointers are refused. It is collected last so
that a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import wavelets as wav
from paper_1801_02417_gb300 import _build
from paper_1801_02417_gb300 import binding as B

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the SARA operator tolerance of the parity tests


@pytest.fixture(scope="module")
def lib():
    _build.build_library()
    return B.lib()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (16, 4): the small-level kernel at the finest level and a fused tail of three levels;
# (128, 4): tiled levels 128 and 64, the small-level kernel at 32 and 16;
# (256, 6): the scratch's largest image, tiled levels 256..64 and a fused tail of three levels.
@pytest.mark.parametrize("n,levels", [(16, 4), (128, 4), (256, 6)])
def test_static_scratch_synthesis_matches_handle_path_and_oracle(lib, n, levels):
    import torch
    cfg = B.ps_config(n=n, levels=levels, mode=0, kernel_width=7)
    h = B.ps_create(cfg)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            A = np.random.default_rng(100 + call).normal(size=(4, 9, n, n)).astype(np.float32)
            expect = np.empty((4, n, n), np.float32)
            B.ps_apply_psi(h, A, expect)
            Ad = torch.from_numpy(A).cuda()
            Sd = torch.full((4, n, n), float("nan"), device="cuda")
            B.ps_apply_psi_static(Ad, Sd, n, levels, stream)
            B.ps_static_status(stream)
            got = Sd.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert _rel(got, expect) <= TOL, (call, _rel(got, expect))
            assert _rel(got, wav.psi(A.astype(np.float64), levels)) <= TOL, call
    finally:
        B.ps_destroy(h)


def test_repeated_call_allocates_nothing(lib):
    import torch
    n, levels = 256, 4
    A = torch.randn(4, 9, n, n, device="cuda")
    S = torch.empty(4, n, n, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    B.ps_apply_psi_static(A, S, n, levels, stream)
    B.ps_static_status(stream)
    first = S.clone()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    reserved1 = torch.cuda.memory_reserved()
    B.ps_apply_psi_static(A, S, n, levels, stream)
    B.ps_static_status(stream)
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1
    assert torch.cuda.memory_reserved() == reserved1
    assert torch.equal(S, first)          # same input through the same scratch: the same result


def test_static_wait_timeout_is_reported(lib):
    """With a zero poll budget the tiled synthesis kernels give up at their first wait (their
    copies are drained before they exit); ps_static_status reports PS_ETIMEOUT, and once the
    budget is restored the next call is complete again."""
    import torch
    n, levels = 128, 2
    A = torch.randn(4, 9, n, n, device="cuda")
    S = torch.empty(4, n, n, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    B.ps_debug_set_wait_polls(0)
    try:
        B.ps_apply_psi_static(A, S, n, levels, stream)
        with pytest.raises(B.PolsaraError) as e:
            B.ps_static_status(stream)
        assert e.value.status == B.PS_ETIMEOUT
    finally:
        B.ps_debug_set_wait_polls(-1)
    B.ps_apply_psi_static(A, S, n, levels, stream)
    B.ps_static_status(stream)
    ref = wav.psi(A.cpu().numpy().astype(np.float64), levels)
    assert _rel(S.cpu().numpy(), ref) <= TOL


def test_static_scratch_rejects_sizes_beyond_its_limit_and_host_pointers(lib):
    import torch
    A = torch.zeros(16, device="cuda")
    S = torch.zeros(16, device="cuda")
    with pytest.raises(B.PolsaraError) as e:
        B.ps_apply_psi_static(A, S, 512, 4)
    assert e.value.status == B.PS_EINVAL
    assert "static scratch" in B.ps_last_error(None)
    # Host memory through the C ABI: refused before any launch.
    n = 16
    Ah = np.zeros((4, 9, n, n), np.float32)
    Sh = np.zeros((4, n, n), np.float32)
    st = lib.ps_apply_psi_static(ctypes.c_void_p(Ah.ctypes.data), ctypes.c_void_p(Sh.ctypes.data), n, 2, None)
    assert st == B.PS_EINVAL
    assert "device" in B.ps_last_error(None)
