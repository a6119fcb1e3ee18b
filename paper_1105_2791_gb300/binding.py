"""Thin ctypes binding of the modal C ABI (include/modal.h).

Each function has the name of the C entry point and only marshals arguments:
host arrays are numpy float64/float32 arrays, device buffers are CUDA torch
tensors (or raw integer device addresses), `stream` defaults to torch's
current stream.  Every computation runs in the CUDA library; there is no CPU
fallback, and importing this module raises if the library is not built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_float, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

from . import build as _build

MODAL_OK, MODAL_EINVAL, MODAL_ENOMEM, MODAL_ECUDA, MODAL_ENOTPD, MODAL_ETIMEOUT, MODAL_ESTATE, MODAL_ENOCONV = range(8)
MODAL_FP32, MODAL_3XTF32, MODAL_BF16X3, MODAL_BF16, MODAL_FP16X3 = range(5)
PREC = {"fp32": MODAL_FP32, "3xtf32": MODAL_3XTF32, "bf16x3": MODAL_BF16X3, "bf16": MODAL_BF16,
        "fp16x3": MODAL_FP16X3}
STATUS_NAMES = ["MODAL_OK", "MODAL_EINVAL", "MODAL_ENOMEM", "MODAL_ECUDA", "MODAL_ENOTPD",
                "MODAL_ETIMEOUT", "MODAL_ESTATE", "MODAL_ENOCONV"]

# Every symbol include/modal.h declares.
EXPORTS = [
    "modal_init", "modal_synthesize", "modal_analyze", "modal_linear_term", "modal_cubic",
    "modal_cov_accumulate", "modal_solve", "modal_backward", "modal_alpha_local", "modal_get_info",
    "modal_get_rings", "modal_get_pair_mean", "modal_get_zeta", "modal_reset", "modal_set_chunk",
    "modal_sync", "modal_save_state", "modal_load_state", "modal_selftest_wait", "modal_destroy",
    "modal_last_error", "modal_set_profiling", "modal_get_profile", "modal_stage_name", "modal_cubic_static",
    "modal_batch_create", "modal_batch_cubic", "modal_batch_destroy", "modal_set_linear_mode",
    "modal_bivector_fit", "modal_solve_bivector", "modal_bivector_rotate", "modal_quartic",
    "modal_set_retain_maps", "modal_backward_retained", "modal_fnl_weights", "modal_peak_probe",
    "modal_get_tuning", "modal_set_tuning", "modal_autotune", "modal_cubic_retained", "modal_batch_set_schedule",
]
MODAL_NSTAGES = 15


class ModalError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message))


class modal_grid(ctypes.Structure):
    _fields_ = [("nrings", c_int), ("nphi", c_int), ("ring_mask", c_void_p), ("pix_mask", c_void_p)]


class modal_info(ctypes.Structure):
    _fields_ = [("lmax", c_int), ("P", c_int), ("nrings", c_int), ("nphi", c_int), ("prec", c_int),
                ("n_alm", c_int), ("n_max", c_int), ("n_pair", c_int), ("npix", c_longlong),
                ("n_lin", c_longlong), ("n_cov", c_longlong), ("lin_final", c_int), ("chunk", c_int),
                ("device_bytes", c_size_t), ("n_quad", c_int)]


class modal_tuning(ctypes.Structure):
    _fields_ = [("chunk", c_int), ("legendre_maps", c_int), ("cubic_ctas", c_int), ("ms", c_float)]


TUNING_FIELDS = ("chunk", "legendre_maps", "cubic_ctas")

_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load the in-tree libmodal.so (raises ImportError if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("modal CUDA library not built (%s); run paper_1105_2791_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    H = c_void_p
    sig = {
        "modal_init": [c_int, c_int, c_void_p, c_void_p, POINTER(modal_grid), c_int, POINTER(H)],
        "modal_synthesize": [H, c_void_p, c_int, c_void_p, c_void_p],
        "modal_analyze": [H, c_void_p, c_int, c_void_p, c_void_p],
        "modal_linear_term": [H, c_void_p, c_int, c_int, c_void_p],
        "modal_cubic": [H, c_void_p, c_int, c_int, c_void_p, c_void_p],
        "modal_cubic_retained": [H, c_void_p, c_int, c_int, c_void_p, c_void_p],
        "modal_cov_accumulate": [H, c_void_p, c_int, c_void_p],
        "modal_solve": [H, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p],
        "modal_fnl_weights": [H, c_void_p, c_void_p, c_void_p, c_void_p],
        "modal_peak_probe": [c_int, c_void_p, c_void_p],
        "modal_get_tuning": [H, POINTER(modal_tuning)],
        "modal_set_tuning": [H, POINTER(modal_tuning)],
        "modal_autotune": [H, c_void_p, c_int, c_int, POINTER(modal_tuning), c_void_p],
        "modal_bivector_fit": [H, c_void_p, c_void_p, c_void_p, c_void_p],
        "modal_solve_bivector": [H, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p],
        "modal_bivector_rotate": [H, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p],
        "modal_quartic": [H, c_void_p, c_int, c_int, c_void_p, c_void_p],
        "modal_backward": [H, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p],
        "modal_backward_retained": [H, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p],
        "modal_set_retain_maps": [H, c_int],
        "modal_alpha_local": [H, c_void_p, c_void_p],
        "modal_get_info": [H, POINTER(modal_info)],
        "modal_get_rings": [H, c_void_p, c_void_p],
        "modal_get_pair_mean": [H, c_void_p, c_void_p],
        "modal_get_zeta": [H, c_void_p],
        "modal_reset": [H, c_int],
        "modal_set_chunk": [H, c_int],
        "modal_sync": [H, c_void_p],
        "modal_save_state": [H, c_char_p],
        "modal_load_state": [H, c_char_p],
        "modal_selftest_wait": [H, c_int, c_void_p],
        "modal_set_profiling": [H, c_int],
        "modal_get_profile": [H, c_void_p, c_void_p, c_int],
        "modal_cubic_static": [c_void_p, c_void_p, c_longlong, c_int, c_int, c_void_p, c_void_p],
        "modal_batch_create": [c_void_p, c_int, POINTER(c_void_p)],
        "modal_set_linear_mode": [H, c_int],
        "modal_batch_cubic": [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p],
        "modal_batch_set_schedule": [c_void_p, c_int],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c_int
    lib.modal_destroy.argtypes = [H]
    lib.modal_destroy.restype = None
    lib.modal_batch_destroy.argtypes = [c_void_p]
    lib.modal_batch_destroy.restype = None
    lib.modal_stage_name.argtypes = [c_int]
    lib.modal_stage_name.restype = c_char_p
    lib.modal_last_error.argtypes = []
    lib.modal_last_error.restype = c_char_p
    _LIB = lib
    return lib


def _check(status: int):
    if status != MODAL_OK:
        msg = load_library().modal_last_error()
        raise ModalError(status, msg.decode() if msg else "")


def _dev(t):
    """Device address of a CUDA tensor (must be contiguous) or a raw integer address."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(c_void_p)


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------ entry points

def modal_init(lmax, P, basis, C_l, nrings, nphi, prec=MODAL_FP32, ring_mask=None, pix_mask=None):
    lib = load_library()
    b_arr, b_ptr = _host(basis, np.float64)
    c_arr, c_ptr = _host(C_l, np.float64)
    rm_arr, rm_ptr = _host(ring_mask, np.float32)
    pm_arr, pm_ptr = _host(pix_mask, np.float32)
    grid = modal_grid(int(nrings), int(nphi), rm_ptr, pm_ptr)
    h = c_void_p()
    _check(lib.modal_init(int(lmax), int(P), b_ptr, c_ptr, byref(grid), int(PREC.get(prec, prec)), byref(h)))
    return h


def modal_synthesize(h, alm, B, maps, stream=None):
    _check(load_library().modal_synthesize(h, _dev(alm), int(B), _dev(maps), _stream(stream)))


def modal_analyze(h, maps, B, alm, stream=None):
    _check(load_library().modal_analyze(h, _dev(maps), int(B), _dev(alm), _stream(stream)))


def modal_linear_term(h, alm_sims, B, finalize, stream=None):
    _check(load_library().modal_linear_term(h, _dev(alm_sims), int(B), int(bool(finalize)), _stream(stream)))


def modal_cubic(h, alm, B, use_linear, beta, stream=None):
    _check(load_library().modal_cubic(h, _dev(alm), int(B), int(bool(use_linear)), _dev(beta), _stream(stream)))


def modal_cubic_retained(h, alm, B, use_linear, beta, stream=None):
    _check(load_library().modal_cubic_retained(h, _dev(alm), int(B), int(bool(use_linear)), _dev(beta),
                                               _stream(stream)))


def modal_quartic(h, alm, B, use_linear, tau, stream=None):
    _check(load_library().modal_quartic(h, _dev(alm), int(B), int(bool(use_linear)), _dev(tau), _stream(stream)))


LINEAR_MODES = {"pixel": 0, "ring": 1}


def modal_set_linear_mode(h, mode):
    """mode: "pixel" (per-pixel Monte Carlo pair means) or "ring" (per-ring means)."""
    _check(load_library().modal_set_linear_mode(h, LINEAR_MODES[mode]))


def modal_batch_create(plans):
    """plans: sequence of plan handles -> batch handle."""
    arr = (c_void_p * len(plans))(*plans)
    out = c_void_p()
    _check(load_library().modal_batch_create(arr, len(plans), byref(out)))
    return out.value


def modal_batch_cubic(bh, alms, Bs, use_linear, betas, use_graph=True, stream=None):
    """alms, Bs, betas: one entry per plan of the batch (device tensors or addresses)."""
    n = len(Bs)
    a = (c_void_p * n)(*[_dev(x) for x in alms])
    b = (c_int * n)(*[int(x) for x in Bs])
    o = (c_void_p * n)(*[_dev(x) for x in betas])
    _check(load_library().modal_batch_cubic(bh, a, b, int(bool(use_linear)), o, int(bool(use_graph)),
                                            _stream(stream)))


BATCH_SCHEDULES = {"streams": 0, "shared_cubic": 1}


def modal_batch_set_schedule(bh, schedule):
    _check(load_library().modal_batch_set_schedule(bh, BATCH_SCHEDULES[schedule]
                                                   if isinstance(schedule, str) else int(schedule)))


def modal_batch_destroy(bh):
    load_library().modal_batch_destroy(bh)


def modal_cov_accumulate(h, beta, B, stream=None):
    _check(load_library().modal_cov_accumulate(h, _dev(beta), int(B), _stream(stream)))


def modal_solve(h, alpha, beta, B, stream=None):
    """Returns (fnl [B] numpy, sigma)."""
    a_arr, a_ptr = _host(alpha, np.float64)
    fnl = np.zeros(max(int(B), 1))
    sigma = c_double(0.0)
    _check(load_library().modal_solve(h, a_ptr, _dev(beta), int(B), fnl.ctypes.data_as(c_void_p), byref(sigma),
                                      _stream(stream)))
    return fnl[: int(B)], sigma.value


def modal_fnl_weights(h, alpha, w, stream=None):
    """w = d fNL / d beta = zeta^-1 alpha / (alpha^T zeta^-1 alpha) into dev w [n_max] float64;
    returns sigma."""
    a_arr, a_ptr = _host(alpha, np.float64)
    sigma = c_double(0.0)
    _check(load_library().modal_fnl_weights(h, a_ptr, _dev(w), byref(sigma), _stream(stream)))
    return sigma.value


PEAK_KINDS = {"fp32_simt": 0, "fp64_simt": 1, "tf32_tensor": 2, "f16_tensor": 3, "tf32_tensor_n16": 4}


def _tuning_dict(t):
    return {"chunk": t.chunk, "legendre_maps": t.legendre_maps, "cubic_ctas": t.cubic_ctas, "ms": float(t.ms)}


def modal_get_tuning(h):
    """The plan's launch shapes as a dict (modal_tuning)."""
    t = modal_tuning()
    _check(load_library().modal_get_tuning(h, byref(t)))
    return _tuning_dict(t)


def modal_set_tuning(h, tuning):
    """Set the launch shapes from a dict with the keys of TUNING_FIELDS."""
    t = modal_tuning(*(int(tuning[k]) for k in TUNING_FIELDS), 0.0)
    _check(load_library().modal_set_tuning(h, byref(t)))


def modal_autotune(h, alm, B, use_linear=False, stream=None):
    """Time candidate launch shapes on the caller's maps; returns the winner (dict, with ms)."""
    t = modal_tuning()
    _check(load_library().modal_autotune(h, _dev(alm), int(B), int(bool(use_linear)), byref(t), _stream(stream)))
    return _tuning_dict(t)


def modal_peak_probe(kind, stream=None):
    """Measured throughput (TFLOP/s) of one of PEAK_KINDS on the current device."""
    v = c_double(0.0)
    _check(load_library().modal_peak_probe(int(PEAK_KINDS.get(kind, kind)), byref(v), _stream(stream)))
    return v.value


def modal_bivector_fit(h, zeta0, stream=None):
    """Returns (bt [n_max] numpy, lambda1)."""
    info = modal_get_info(h)
    z_arr, z_ptr = _host(zeta0, np.float64)
    bt = np.zeros(info.n_max)
    lam = c_double(0.0)
    _check(load_library().modal_bivector_fit(h, z_ptr, bt.ctypes.data_as(c_void_p), byref(lam), _stream(stream)))
    return bt, lam.value


def modal_solve_bivector(h, zeta0, bt, alpha, beta, B, stream=None):
    """Returns (fnl [B] numpy, sigma)."""
    z_arr, z_ptr = _host(zeta0, np.float64)
    b_arr, b_ptr = _host(bt, np.float64)
    a_arr, a_ptr = _host(alpha, np.float64)
    fnl = np.zeros(max(int(B), 1))
    sigma = c_double(0.0)
    _check(load_library().modal_solve_bivector(h, z_ptr, b_ptr, a_ptr, _dev(beta), int(B),
                                               fnl.ctypes.data_as(c_void_p), byref(sigma), _stream(stream)))
    return fnl[: int(B)], sigma.value


def modal_bivector_rotate(h, zeta0, bt, x, B, out, stream=None):
    z_arr, z_ptr = _host(zeta0, np.float64)
    b_arr, b_ptr = _host(bt, np.float64)
    _check(load_library().modal_bivector_rotate(h, z_ptr, b_ptr, _dev(x), int(B), _dev(out), _stream(stream)))


def modal_backward(h, alm, B, g, use_linear, grad_alm, stream=None):
    _check(load_library().modal_backward(h, _dev(alm), int(B), _dev(g), int(bool(use_linear)), _dev(grad_alm),
                                         _stream(stream)))


def modal_set_retain_maps(h, on):
    _check(load_library().modal_set_retain_maps(h, int(bool(on))))


def modal_backward_retained(h, alm, B, g, use_linear, grad_alm, stream=None):
    _check(load_library().modal_backward_retained(h, _dev(alm), int(B), _dev(g), int(bool(use_linear)),
                                                  _dev(grad_alm), _stream(stream)))


def modal_alpha_local(h, C_signal=None):
    info = modal_get_info(h)
    out = np.zeros(info.n_max)
    c_arr, c_ptr = _host(C_signal, np.float64)
    _check(load_library().modal_alpha_local(h, c_ptr, out.ctypes.data_as(c_void_p)))
    return out


def modal_get_info(h) -> modal_info:
    info = modal_info()
    _check(load_library().modal_get_info(h, byref(info)))
    return info


def modal_get_rings(h):
    n = modal_get_info(h).nrings
    mu, w = np.zeros(n), np.zeros(n)
    _check(load_library().modal_get_rings(h, mu.ctypes.data_as(c_void_p), w.ctypes.data_as(c_void_p)))
    return mu, w


def modal_get_pair_mean(h, out, stream=None):
    _check(load_library().modal_get_pair_mean(h, _dev(out), _stream(stream)))


def modal_get_zeta(h):
    n = modal_get_info(h).n_max
    z = np.zeros((n, n))
    _check(load_library().modal_get_zeta(h, z.ctypes.data_as(c_void_p)))
    return z


def modal_reset(h, what):
    _check(load_library().modal_reset(h, int(what)))


def modal_set_chunk(h, chunk):
    _check(load_library().modal_set_chunk(h, int(chunk)))


def modal_sync(h, stream=None):
    _check(load_library().modal_sync(h, _stream(stream)))


def modal_save_state(h, path):
    _check(load_library().modal_save_state(h, str(path).encode()))


def modal_load_state(h, path):
    _check(load_library().modal_load_state(h, str(path).encode()))


def modal_selftest_wait(h, spin_limit, stream=None):
    _check(load_library().modal_selftest_wait(h, int(spin_limit), _stream(stream)))


def modal_set_profiling(h, enable):
    _check(load_library().modal_set_profiling(h, int(bool(enable))))


def modal_get_profile(h):
    """{stage name: (ms, launches)} accumulated since the previous call (then reset)."""
    ms = np.zeros(MODAL_NSTAGES)
    n = np.zeros(MODAL_NSTAGES, dtype=np.int64)
    _check(load_library().modal_get_profile(h, ms.ctypes.data_as(c_void_p), n.ctypes.data_as(c_void_p),
                                            MODAL_NSTAGES))
    return {modal_stage_name(i): (float(ms[i]), int(n[i])) for i in range(MODAL_NSTAGES)}


def modal_stage_name(stage):
    return load_library().modal_stage_name(int(stage)).decode()


def modal_cubic_static(maps, W, npix, P, B, beta, stream=None):
    """Allocation-free cubic coefficients of caller-held maps (see include/modal.h).

    Tensors are checked before the call (the library sees raw pointers only): maps float32
    with at least B * P * npix elements, W float32 with at least npix, beta float64 with at
    least B * n_max, all contiguous on the current CUDA device."""
    import torch
    npix, P, B = int(npix), int(P), int(B)
    n_max = P * (P + 1) * (P + 2) // 6
    dev = torch.cuda.current_device()
    for name, t, dtype, need in (("maps", maps, torch.float32, B * P * npix), ("W", W, torch.float32, npix),
                                 ("beta", beta, torch.float64, B * n_max)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a CUDA tensor" % name)
        if not t.is_cuda or t.device.index != dev:
            raise ValueError("%s must be on the current CUDA device (cuda:%d)" % (name, dev))
        if t.dtype != dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if t.numel() < need:
            raise ValueError("%s holds %d elements, the call reads or writes %d" % (name, t.numel(), need))
    _check(load_library().modal_cubic_static(_dev(maps), _dev(W), npix, P, B, _dev(beta), _stream(stream)))


def modal_destroy(h):
    if h is not None and h.value:
        load_library().modal_destroy(h)


def modal_last_error() -> str:
    msg = load_library().modal_last_error()
    return msg.decode() if msg else ""
