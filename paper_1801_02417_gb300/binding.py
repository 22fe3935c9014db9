"""Thin ctypes binding of the C ABI in include/polsara.h (argument marshalling only).

Each function has the name of the C entry point it calls. Array arguments may be
numpy arrays (host memory) or torch CUDA tensors (device memory, used on the
handle's stream); the `device_ptrs` flag of the C call is derived from the
argument. Every non-zero status raises PolsaraError with ps_last_error().
The CUDA library must be built (``paper_1801_02417_gb300._build.build_library``);
there is no fallback: importing a function without the library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

PS_OK, PS_EINVAL, PS_ENOMEM, PS_ECUDA, PS_ETIMEOUT, PS_ENONFINITE, PS_ESTATE = range(7)
PS_POLARIZED, PS_NO_CONSTRAINT, PS_NNLS, PS_SOC = 0, 1, 2, 3
PS_TV, PS_TV_NC, PS_L1TV, PS_L1TV_NC = 4, 5, 6, 7
PS_STOP_REL, PS_STOP_RESID, PS_STOP_NP = 1, 2, 4
STATUS_NAMES = {0: "PS_OK", 1: "PS_EINVAL", 2: "PS_ENOMEM", 3: "PS_ECUDA", 4: "PS_ETIMEOUT",
                5: "PS_ENONFINITE", 6: "PS_ESTATE"}


class PolsaraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ps_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("levels", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("literal_ball", ctypes.c_int32), ("kernel_width", ctypes.c_int32),
                ("stop_maps", ctypes.c_int32), ("tau", ctypes.c_double), ("rho1", ctypes.c_double),
                ("rho2", ctypes.c_double), ("rho3", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gamma", ctypes.c_double), ("noise_sigma", ctypes.c_double), ("rel_tol", ctypes.c_double),
                ("resid_tol", ctypes.c_double), ("np_tol", ctypes.c_double), ("zeta_sigma", ctypes.c_double)]


class ps_stats(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int32), ("stop_flags", ctypes.c_int32),
                ("block_residual", ctypes.POINTER(ctypes.c_double)), ("rel_change", ctypes.c_double * 4),
                ("zeta", ctypes.c_double), ("violations", ctypes.c_int64), ("violations_raw", ctypes.c_int64),
                ("weighted_l1", ctypes.c_double), ("iterations", ctypes.c_int64), ("converged", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ps_state_view(ctypes.Structure):
    _fields_ = [("S", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("D", ctypes.c_void_p), ("device_ptrs", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I32, _I64, _F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double

_SIGS = {
    "ps_create": (_I32, [ctypes.POINTER(ps_config), _P, ctypes.POINTER(_H)]),
    "ps_destroy": (None, [_H]),
    "ps_last_error": (ctypes.c_char_p, [_H]),
    "ps_set_measurements": (_I32, [_H, _I64, _P, _P, _P, _I32, _P, _P, _I32]),
    "ps_set_sara_weights": (_I32, [_H, _P, _F64, _I32]),
    "ps_get_sara_weights": (_I32, [_H, _P, _I32]),
    "ps_pd_iterate": (_I32, [_H, _I32, ctypes.POINTER(ps_stats)]),
    "ps_reweight": (_I32, [_H, _F64]),
    "ps_set_mode": (_I32, [_H, _I32]),
    "ps_set_tv_weights": (_I32, [_H, _P, _P]),
    "ps_get_stokes": (_I32, [_H, _P, _I32]),
    "ps_get_state": (_I32, [_H, ctypes.POINTER(ps_state_view)]),
    "ps_set_state": (_I32, [_H, ctypes.POINTER(ps_state_view)]),
    "ps_get_params": (_I32, [_H] + [ctypes.POINTER(_F64)] * 5),
    "ps_get_config": (_I32, [_H, ctypes.POINTER(ps_config)]),
    "ps_compute_stats": (_I32, [_H, _F64, ctypes.POINTER(ps_stats)]),
    "ps_apply_phi": (_I32, [_H, _P, _P, _I32]),
    "ps_apply_phi_adjoint": (_I32, [_H, _P, _P, _I32]),
    "ps_apply_psi_adjoint": (_I32, [_H, _P, _P, _I32]),
    "ps_apply_psi": (_I32, [_H, _P, _P, _I32]),
    "ps_wavelet_filters": (_I32, [_P]),
    "ps_apply_psi_static": (_I32, [_P, _P, _I32, _I32, _P]),
    "ps_static_status": (_I32, [_P]),
    "ps_debug_set_wait_polls": (_I32, [_I32]),
    "ps_fp32_peak": (_I32, [_I32, ctypes.POINTER(_F64)]),
    "ps_set_visibilities": (_I32, [_H, _P, _I32]),
    "ps_get_rel_change": (_I32, [_H, _P]),
    "ps_rel_change_request": (_I32, [_H]),
    "ps_rel_change_result": (_I32, [_H, _P]),
    "ps_max_abs_analysis": (_I32, [_H, ctypes.POINTER(_F64)]),
    "ps_batch_create": (_I32, [_P, _I32, _P, ctypes.POINTER(_H)]),
    "ps_batch_iterate": (_I32, [_H, _I32]),
    "ps_batch_synchronize": (_I32, [_H]),
    "ps_batch_destroy": (None, [_H]),
    "ps_profile_stages": (_I32, [_H, _I32, _P]),
    "ps_kernels_per_iteration": (_I32, [_H]),
    "ps_synchronize": (_I32, [_H]),
    "ps_device_bytes": (_I64, [_H]),
    "ps_estimate_bytes": (_I64, [_I32, _I32, _I64]),
    "ps_autotune": (_I32, [_H, _I32, _P, _P]),
    "ps_get_tuning": (_I32, [_H, _P]),
    "ps_set_tuning": (_I32, [_H, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libpolsara.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1801_02417_gb300._build.build_library()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(h, status: int) -> None:
    if status != PS_OK:
        msg = lib().ps_last_error(h)
        raise PolsaraError(status, msg.decode() if msg else "")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arg(x, dtype, writable=False):
    """(pointer, device flag, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError(f"output arrays must be C-contiguous {dtype}")
        a = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def ps_create(cfg: ps_config, stream=None):
    h = _H()
    s = ctypes.c_void_p(int(stream)) if stream else None
    st = lib().ps_create(ctypes.byref(cfg), s, ctypes.byref(h))
    _check(None, st)
    return h


def ps_destroy(h) -> None:
    lib().ps_destroy(h)


def ps_last_error(h) -> str:
    msg = lib().ps_last_error(h)
    return msg.decode() if msg else ""


def ps_set_measurements(h, uv, vis, weights, block_offsets, eps) -> None:
    """eps None: the chi^2 radii from the handle's noise_sigma."""
    puv, d1, k1 = _arg(uv, np.float64)
    pv, d2, k2 = _arg(vis, np.complex64)
    pw, d3, k3 = _arg(weights, np.float32)
    off = np.ascontiguousarray(block_offsets, dtype=np.int64)
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    dev = d1 or d2 or d3
    if weights is not None and d3 != dev or d1 != d2:
        raise ValueError("uv, vis and weights must all be host arrays or all device tensors")
    M = int(uv.shape[0])
    nb = len(off) - 1 if e is None else len(e)
    _check(h, lib().ps_set_measurements(h, M, puv, pv, pw, nb, ctypes.c_void_p(off.ctypes.data),
                                        None if e is None else ctypes.c_void_p(e.ctypes.data), dev))


def ps_set_sara_weights(h, W, gamma: float) -> None:
    p, d, k = _arg(W, np.float32)
    _check(h, lib().ps_set_sara_weights(h, p, float(gamma), d))


def ps_get_sara_weights(h, out) -> None:
    p, d, k = _arg(out, np.float32, writable=True)
    _check(h, lib().ps_get_sara_weights(h, p, d))


def ps_pd_iterate(h, n_iter: int, stats_nblocks: int | None = None):
    """n_iter iterations; with stats_nblocks (the handle's block count) also returns the
    stopping-rule statistics of the new state (a dict as ps_compute_stats)."""
    if stats_nblocks is None:
        _check(h, lib().ps_pd_iterate(h, int(n_iter), None))
        return None
    st, res = _stats_struct(stats_nblocks)
    _check(h, lib().ps_pd_iterate(h, int(n_iter), ctypes.byref(st)))
    return _stats_dict(st, res, stats_nblocks)


def ps_reweight(h, delta: float) -> None:
    _check(h, lib().ps_reweight(h, float(delta)))


def ps_set_mode(h, mode: int) -> None:
    _check(h, lib().ps_set_mode(h, int(mode)))


def ps_set_tv_weights(h, tv, l1=None) -> None:
    """TV weights mu_i (and l1 weights nu_i) per Stokes map I, Q, U, V (Algorithm 3)."""
    t = np.ascontiguousarray(np.asarray(tv, dtype=np.float64).reshape(4))
    a = None if l1 is None else np.ascontiguousarray(np.asarray(l1, dtype=np.float64).reshape(4))
    _check(h, lib().ps_set_tv_weights(h, ctypes.c_void_p(t.ctypes.data),
                                      ctypes.c_void_p(a.ctypes.data) if a is not None else None))


def ps_get_stokes(h, out) -> None:
    p, d, k = _arg(out, np.float32, writable=True)
    _check(h, lib().ps_get_stokes(h, p, d))


def _view(arrays: dict, writable: bool):
    v = ps_state_view()
    keep = []
    dev = None
    dtypes = {"B": np.complex64}
    for name in ("S", "Z", "A", "B", "C", "D"):
        x = arrays.get(name)
        if x is None:
            continue
        p, d, k = _arg(x, dtypes.get(name, np.float32), writable)
        if dev is not None and d != dev:
            raise ValueError("state arrays must all be host arrays or all device tensors")
        dev = d
        setattr(v, name, p)
        keep.append(k)
    v.device_ptrs = dev or 0
    return v, keep


def ps_get_state(h, arrays: dict) -> None:
    v, keep = _view(arrays, True)
    _check(h, lib().ps_get_state(h, ctypes.byref(v)))


def ps_set_state(h, arrays: dict) -> None:
    v, keep = _view(arrays, False)
    _check(h, lib().ps_set_state(h, ctypes.byref(v)))


def ps_get_params(h) -> dict:
    vals = [_F64() for _ in range(5)]
    _check(h, lib().ps_get_params(h, *[ctypes.byref(v) for v in vals]))
    return dict(zip(("tau", "rho1", "rho2", "rho3", "opnorm_sq"), (v.value for v in vals)))


def _stats_struct(nblocks: int):
    res = (ctypes.c_double * max(1, nblocks))()
    st = ps_stats()
    st.nblocks = nblocks
    st.block_residual = ctypes.cast(res, ctypes.POINTER(ctypes.c_double))
    return st, res


def _stats_dict(st, res, nblocks: int) -> dict:
    return {"block_residual": np.array(res[:nblocks]), "rel_change": np.array(st.rel_change[:]),
            "zeta": st.zeta, "violations": st.violations, "violations_raw": st.violations_raw,
            "weighted_l1": st.weighted_l1, "iterations": st.iterations, "stop_flags": st.stop_flags,
            "converged": bool(st.converged)}


def ps_get_config(h) -> ps_config:
    cfg = ps_config()
    _check(h, lib().ps_get_config(h, ctypes.byref(cfg)))
    return cfg


def ps_compute_stats(h, zeta_sigma: float, nblocks: int) -> dict:
    """Stopping-rule statistics (zeta_sigma <= 0: the handle's)."""
    st, res = _stats_struct(nblocks)
    _check(h, lib().ps_compute_stats(h, float(zeta_sigma), ctypes.byref(st)))
    return _stats_dict(st, res, nblocks)


def _op(name, h, x, out, in_dtype, out_dtype):
    px, dx, kx = _arg(x, in_dtype)
    po, do, ko = _arg(out, out_dtype, writable=True)
    if dx != do:
        raise ValueError("input and output must both be host arrays or both device tensors")
    _check(h, getattr(lib(), name)(h, px, po, dx))


def ps_apply_phi(h, S, Y) -> None:
    _op("ps_apply_phi", h, S, Y, np.float32, np.complex64)


def ps_apply_phi_adjoint(h, Y, S) -> None:
    _op("ps_apply_phi_adjoint", h, Y, S, np.complex64, np.float32)


def ps_apply_psi_adjoint(h, S, A) -> None:
    _op("ps_apply_psi_adjoint", h, S, A, np.float32, np.float32)


def ps_apply_psi(h, A, S) -> None:
    _op("ps_apply_psi", h, A, S, np.float32, np.float32)


def ps_apply_psi_static(A, S, n: int, levels: int, stream=None) -> None:
    """Allocation-free Psi A; A and S must be CUDA tensors (device pointers)."""
    pa, da, ka = _arg(A, np.float32)
    ps_, ds, ks = _arg(S, np.float32, writable=True)
    if not (da and ds):
        raise ValueError("ps_apply_psi_static takes device tensors only")
    st = ctypes.c_void_p(int(stream)) if stream else None
    _check(None, lib().ps_apply_psi_static(pa, ps_, int(n), int(levels), st))


def ps_static_status(stream=None) -> None:
    """Raises PolsaraError(PS_ETIMEOUT) if the last ps_apply_psi_static call on this device gave up."""
    st = ctypes.c_void_p(int(stream)) if stream else None
    _check(None, lib().ps_static_status(st))


def ps_debug_set_wait_polls(polls: int) -> None:
    """Test hook: bounded-wait poll budget of every kernel (0: give up at once; < 0: default)."""
    _check(None, lib().ps_debug_set_wait_polls(int(polls)))


def ps_fp32_peak(packed: bool = True) -> float:
    """Measured FP32 FLOP/s of the current device (packed FP32x2 or scalar FMA chains)."""
    v = _F64()
    _check(None, lib().ps_fp32_peak(int(bool(packed)), ctypes.byref(v)))
    return v.value


def ps_wavelet_filters() -> np.ndarray:
    out = np.zeros((8, 16), dtype=np.float64)
    st = lib().ps_wavelet_filters(ctypes.c_void_p(out.ctypes.data))
    _check(None, st)
    return out


def ps_set_visibilities(h, vis) -> None:
    p, d, k = _arg(vis, np.complex64)
    _check(h, lib().ps_set_visibilities(h, p, d))


def ps_get_rel_change(h) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    _check(h, lib().ps_get_rel_change(h, ctypes.c_void_p(out.ctypes.data)))
    return out


def ps_rel_change_request(h) -> None:
    _check(h, lib().ps_rel_change_request(h))


def ps_rel_change_result(h) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    _check(h, lib().ps_rel_change_result(h, ctypes.c_void_p(out.ctypes.data)))
    return out


def ps_max_abs_analysis(h) -> float:
    v = _F64()
    _check(h, lib().ps_max_abs_analysis(h, ctypes.byref(v)))
    return v.value


def ps_batch_create(handles, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = _H()
    s = ctypes.c_void_p(int(stream)) if stream else None
    _check(None, lib().ps_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(handles), s, ctypes.byref(b)))
    return b


def ps_batch_iterate(b, n_iter: int) -> None:
    _check(None, lib().ps_batch_iterate(b, int(n_iter)))


def ps_batch_synchronize(b) -> None:
    _check(None, lib().ps_batch_synchronize(b))


def ps_batch_destroy(b) -> None:
    lib().ps_batch_destroy(b)


STAGES = ("primal", "analysis", "analysis_coarse", "synthesis_coarse", "synthesis", "fwd_fft", "degrid", "ball",
          "grid", "adj_fft")


def ps_profile_stages(h, n_iter: int) -> dict:
    out = np.zeros(len(STAGES), dtype=np.float64)
    _check(h, lib().ps_profile_stages(h, int(n_iter), ctypes.c_void_p(out.ctypes.data)))
    return dict(zip(STAGES, out.tolist()))


def ps_kernels_per_iteration(h) -> int:
    return int(lib().ps_kernels_per_iteration(h))


def ps_synchronize(h) -> None:
    _check(h, lib().ps_synchronize(h))


def ps_device_bytes(h) -> int:
    return int(lib().ps_device_bytes(h))


def ps_estimate_bytes(n: int, levels: int, M: int) -> int:
    return int(lib().ps_estimate_bytes(int(n), int(levels), int(M)))


TUNE_SLOTS = ("synthesis", "degrid", "grid", "analysis")


def ps_autotune(h, reps: int = 5) -> dict:
    """Time every launch candidate on the handle's data and keep the fastest; returns
    {slot: (choice, ms)}."""
    ch = np.zeros(len(TUNE_SLOTS), dtype=np.int32)
    ms = np.zeros(len(TUNE_SLOTS), dtype=np.float64)
    _check(h, lib().ps_autotune(h, int(reps), ctypes.c_void_p(ch.ctypes.data), ctypes.c_void_p(ms.ctypes.data)))
    return {k: (int(c), float(t)) for k, c, t in zip(TUNE_SLOTS, ch, ms)}


def ps_get_tuning(h) -> list:
    ch = np.zeros(len(TUNE_SLOTS), dtype=np.int32)
    _check(h, lib().ps_get_tuning(h, ctypes.c_void_p(ch.ctypes.data)))
    return ch.tolist()


def ps_set_tuning(h, choices) -> None:
    ch = np.ascontiguousarray(choices, dtype=np.int32)
    if ch.size != len(TUNE_SLOTS):
        raise ValueError(f"expected {len(TUNE_SLOTS)} tuning slots")
    _check(h, lib().ps_set_tuning(h, ctypes.c_void_p(ch.ctypes.data)))
