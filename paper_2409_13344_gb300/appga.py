"""Python binding of the APPGA C ABI (``include/appga.h``).

Argument marshalling only: every function here converts its arguments and
calls the C function of the same name in ``libappga.so``; all arithmetic
runs in the library's CUDA kernels.  Device buffers are ``torch`` CUDA
tensors (or raw integer device addresses); streams default to torch's
current stream.  There is no CPU fallback: importing the library fails
loudly when ``libappga.so`` is missing.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libappga.so")

# ---- constants mirrored from appga.h ----
APPGA_OK = 0
APPGA_EINVAL = 1
APPGA_ENOMEM = 2
APPGA_EDOMAIN = 3
APPGA_ETIMEOUT = 4
APPGA_ECUDA = 5
APPGA_ENODEV = 6
APPGA_EBUSY = 7
APPGA_ENUMERIC = 8
APPGA_A_BF16_COPY = 1
APPGA_A_NO_FOLD = 2
APPGA_PREC_FP32 = 0
APPGA_PREC_BF16 = 1
APPGA_MOMENTUM_GN = 0
APPGA_MOMENTUM_NONE = 1
APPGA_MOMENTUM_NESTEROV = 2
APPGA_FLAG_NONFINITE = 1
APPGA_FLAG_TIMEOUT = 2
APPGA_FLAG_DOMAIN = 4


class appga_params(ctypes.Structure):
    _fields_ = [
        ("lambda1", ctypes.c_double), ("lambda2", ctypes.c_double), ("eps", ctypes.c_double),
        ("omega", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("beta", ctypes.c_double), ("max_iters", ctypes.c_int32), ("rel_obj_tol", ctypes.c_double),
        ("precond_freeze_iter", ctypes.c_int32), ("a_precision", ctypes.c_int32),
        ("momentum", ctypes.c_int32), ("track_objective", ctypes.c_int32),
        ("graph_iters", ctypes.c_int32),
    ]


class appga_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("result_k", ctypes.c_int32), ("stopped_early", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("guard_hits", ctypes.c_int64), ("phi", ctypes.c_double),
        ("phi_prev", ctypes.c_double),
    ]


class appga_matrix_info(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int32), ("d", ctypes.c_int32), ("n_side", ctypes.c_int32),
        ("n_angles", ctypes.c_int32), ("nnz", ctypes.c_int64), ("nnz_padded_a", ctypes.c_int64),
        ("nnz_padded_t", ctypes.c_int64), ("has_bf16", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64), ("packed_columns", ctypes.c_int32),
        ("sliced_layout", ctypes.c_int32), ("quarter_turn_folded", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class appga_batch_tuning(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32), ("a_precision", ctypes.c_int32), ("spmv_per_sm", ctypes.c_int32),
        ("stencil_per_sm", ctypes.c_int32), ("pixel_per_sm", ctypes.c_int32),
        ("chunk", ctypes.c_int32), ("gather_rows_fw", ctypes.c_int32),
        ("gather_rows_px", ctypes.c_int32), ("us_per_slice_iter", ctypes.c_double),
        ("us_per_slice_iter_default", ctypes.c_double),
    ]


class appga_afppa_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("flags", ctypes.c_int32), ("guard_hits", ctypes.c_int64),
        ("re", ctypes.c_double), ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
    ]


class appga_fom(ctypes.Structure):
    _fields_ = [
        ("mse", ctypes.c_double), ("psnr", ctypes.c_double), ("rc", ctypes.c_double),
        ("rc_true", ctypes.c_double), ("nrc", ctypes.c_double), ("n_roi_h", ctypes.c_int64),
        ("n_roi_b", ctypes.c_int64),
    ]


class appga_server_config(ctypes.Structure):
    _fields_ = [
        ("slots_per_pool", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32),
        ("a_precision", ctypes.c_int32), ("max_pools", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_int64), ("hbm_reserve_bytes", ctypes.c_int64),
        ("max_pools_per_geometry", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


class appga_request_stats(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32), ("iters", ctypes.c_int32), ("result_k", ctypes.c_int32),
        ("stopped_early", ctypes.c_int32), ("flags", ctypes.c_int32), ("phi_k", ctypes.c_int32),
        ("guard_hits", ctypes.c_int64), ("phi_last", ctypes.c_double),
        ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
    ]


class appga_server_summary(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("waiting", ctypes.c_int64),
        ("running", ctypes.c_int64), ("slice_iters", ctypes.c_int64), ("pools", ctypes.c_int32),
        ("pad", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
        ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
        ("mean_latency_s", ctypes.c_double), ("max_latency_s", ctypes.c_double),
        ("mean_queue_s", ctypes.c_double), ("pool_slot_steps", ctypes.c_int64),
        ("live_slot_steps", ctypes.c_int64), ("replay_seconds", ctypes.c_double),
    ]


APPGA_REQ_WAITING = 0
APPGA_REQ_RUNNING = 1
APPGA_REQ_DONE = 2

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes); the exported surface of appga.h
SIGNATURES = {
    "appga_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "appga_last_error": (ctypes.c_char_p, []),
    "appga_version": (ctypes.c_char_p, []),
    "appga_ctx_create": (ctypes.c_int, [_I32, ctypes.POINTER(_P)]),
    "appga_ctx_destroy": (ctypes.c_int, [_P]),
    "appga_matrix_create": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _P, _P, _P, ctypes.c_uint32,
                                           ctypes.POINTER(_P)]),
    "appga_matrix_destroy": (ctypes.c_int, [_P]),
    "appga_matrix_get_info": (ctypes.c_int, [_P, ctypes.POINTER(appga_matrix_info)]),
    "appga_params_default": (None, [ctypes.POINTER(appga_params)]),
    "appga_params_validate": (ctypes.c_int, [ctypes.POINTER(appga_params)]),
    "appga_gn_theta": (_D, [_I32, _D, _D, _D]),
    "appga_forward_ratio": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "appga_backproject": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "appga_shoitv_grad": (ctypes.c_int, [_P, _I32, _P, _D, _D, _D, _P, _P]),
    "appga_pixel_update": (ctypes.c_int, [_P, _P, _P, _P, _P, _D, ctypes.POINTER(appga_params), _P,
                                          _P]),
    "appga_objective": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(appga_params),
                                       ctypes.POINTER(_D), _P]),
    "appga_initial_image": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "appga_reconstruct": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(appga_params), _P,
                                         ctypes.POINTER(appga_stats), _P]),
    "appga_resume": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _I32, ctypes.POINTER(appga_params), _P,
                                    _P, ctypes.POINTER(appga_stats), _P]),
    "appga_reconstruct_host": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(appga_params), _P,
                                              ctypes.POINTER(appga_stats), _P]),
    "appga_validate_csr_host": (ctypes.c_int, [_I32, _I32, _P, _P, _P]),
    "appga_objective_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(appga_params),
                                               _P, _P]),
    "appga_reconstruct_batched": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P,
                                                 ctypes.POINTER(appga_params), _P,
                                                 ctypes.POINTER(appga_stats), _P]),
    "appga_gather_probe": (ctypes.c_int, [_P, _P, _I32, _I32, ctypes.POINTER(_D),
                                          ctypes.POINTER(_D)]),
    "appga_shoitv3d_grad": (ctypes.c_int, [_P, _I32, _I32, _P, _D, _D, _D, _P, _P, _P]),
    "appga_reconstruct_volume": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P,
                                                ctypes.POINTER(appga_params), _P,
                                                ctypes.POINTER(appga_stats), _P]),
    "appga_kernel_times": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(appga_params), _I32,
                                          ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "appga_autotune_batched": (ctypes.c_int, [_P, _P, _I32, _P, _P, ctypes.POINTER(appga_params),
                                              ctypes.POINTER(appga_batch_tuning)]),
    "appga_batch_schedule_get": (ctypes.c_int, [_P, ctypes.POINTER(appga_batch_tuning)]),
    "appga_batch_schedule_set": (ctypes.c_int, [_P, ctypes.POINTER(appga_batch_tuning)]),
    "appga_afppa_reconstruct": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(appga_params),
                                               _P, _P, _P, ctypes.POINTER(appga_afppa_stats), _P]),
    "appga_figures_of_merit": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _D,
                                              ctypes.POINTER(appga_fom), _P]),
    "appga_nofv": (_D, [_D, _D, _D]),
    "appga_central_line_profile": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    # appga_server.h
    "appga_server_config_default": (None, [ctypes.POINTER(appga_server_config)]),
    "appga_server_create": (ctypes.c_int, [_P, ctypes.POINTER(appga_server_config),
                                           ctypes.POINTER(_P)]),
    "appga_server_destroy": (ctypes.c_int, [_P]),
    "appga_server_add_geometry": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I32)]),
    "appga_server_submit": (ctypes.c_int, [_P, _I32, _P, _P, _P, ctypes.POINTER(appga_params),
                                           ctypes.POINTER(_I64)]),
    "appga_server_step": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "appga_server_poll": (ctypes.c_int, [_P, _I64, ctypes.POINTER(appga_request_stats)]),
    "appga_server_collect": (ctypes.c_int, [_P, _I64, _P, ctypes.POINTER(appga_request_stats)]),
    "appga_server_get_summary": (ctypes.c_int, [_P, ctypes.POINTER(appga_server_summary)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libappga.so (raises if it is missing; there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
            " (the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AppgaError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        msg = lib.appga_last_error().decode()
        super().__init__(f"{where}: {lib.appga_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(rc: int, where: str):
    if rc != APPGA_OK:
        raise AppgaError(rc, where)


def _ptr(x) -> Optional[int]:
    """Device/host address of a tensor (or an int / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_params(**kw) -> appga_params:
    p = appga_params()
    load_library().appga_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"appga_params has no field {k!r}")
        setattr(p, k, v)
    return p


# ---- thin wrappers with the C names ----

def appga_ctx_create(device: int = 0) -> int:
    h = _P()
    _check(load_library().appga_ctx_create(device, ctypes.byref(h)), "appga_ctx_create")
    return h.value


def appga_ctx_destroy(ctx: int):
    _check(load_library().appga_ctx_destroy(ctx), "appga_ctx_destroy")


def appga_matrix_create(ctx: int, m: int, d: int, n_side: int, n_angles: int, row_ptr, col, val,
                        flags: int = 0) -> int:
    """row_ptr/col/val: contiguous host numpy arrays (int32, int32, float32)."""
    import numpy as np
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    h = _P()
    _check(load_library().appga_matrix_create(
        ctx, m, d, n_side, n_angles, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
        flags, ctypes.byref(h)), "appga_matrix_create")
    return h.value


def appga_matrix_destroy(mat: int):
    _check(load_library().appga_matrix_destroy(mat), "appga_matrix_destroy")


def appga_matrix_get_info(mat: int) -> appga_matrix_info:
    info = appga_matrix_info()
    _check(load_library().appga_matrix_get_info(mat, ctypes.byref(info)), "appga_matrix_get_info")
    return info


def appga_params_validate(p: appga_params) -> int:
    return load_library().appga_params_validate(ctypes.byref(p))


def appga_gn_theta(k: int, a: float, b: float, omega: float) -> float:
    return load_library().appga_gn_theta(k, a, b, omega)


def appga_forward_ratio(ctx, mat, f, g, gamma, y_out, w_out=None, data_out=None, stream=None):
    _check(load_library().appga_forward_ratio(ctx, mat, _ptr(f), _ptr(g), _ptr(gamma), _ptr(y_out),
                                              _ptr(w_out), _ptr(data_out), _stream(stream)),
           "appga_forward_ratio")


def appga_backproject(ctx, mat, w, out, stream=None):
    _check(load_library().appga_backproject(ctx, mat, _ptr(w), _ptr(out), _stream(stream)),
           "appga_backproject")


def appga_shoitv_grad(ctx, n_side, f, lambda1, lambda2, eps, out, stream=None):
    _check(load_library().appga_shoitv_grad(ctx, n_side, _ptr(f), lambda1, lambda2, eps, _ptr(out),
                                            _stream(stream)), "appga_shoitv_grad")


def appga_pixel_update(ctx, mat, f_prev, f_cur, w, theta, params, f_next, stream=None):
    _check(load_library().appga_pixel_update(ctx, mat, _ptr(f_prev), _ptr(f_cur), _ptr(w), theta,
                                             ctypes.byref(params), _ptr(f_next), _stream(stream)),
           "appga_pixel_update")


def appga_objective(ctx, mat, f, g, gamma, params, stream=None) -> float:
    out = ctypes.c_double()
    _check(load_library().appga_objective(ctx, mat, _ptr(f), _ptr(g), _ptr(gamma),
                                          ctypes.byref(params), ctypes.byref(out), _stream(stream)),
           "appga_objective")
    return out.value


def appga_initial_image(ctx, mat, g, gamma, f_out, stream=None):
    _check(load_library().appga_initial_image(ctx, mat, _ptr(g), _ptr(gamma), _ptr(f_out),
                                              _stream(stream)), "appga_initial_image")


def appga_reconstruct(ctx, mat, g, gamma, f_init, params, f_out, stream=None) -> appga_stats:
    st = appga_stats()
    _check(load_library().appga_reconstruct(ctx, mat, _ptr(g), _ptr(gamma), _ptr(f_init),
                                            ctypes.byref(params), _ptr(f_out), ctypes.byref(st),
                                            _stream(stream)), "appga_reconstruct")
    return st


def appga_resume(ctx, mat, g, gamma, f_prev, f_cur, k0, params, f_out_prev, f_out,
                 stream=None) -> appga_stats:
    st = appga_stats()
    _check(load_library().appga_resume(ctx, mat, _ptr(g), _ptr(gamma), _ptr(f_prev), _ptr(f_cur),
                                       k0, ctypes.byref(params), _ptr(f_out_prev), _ptr(f_out),
                                       ctypes.byref(st), _stream(stream)), "appga_resume")
    return st


def appga_reconstruct_host(ctx, mat, g_host, gamma_host, f_init_host, params, f_out_host,
                           stream=None) -> appga_stats:
    """Host buffers: numpy arrays or (pinned) CPU torch tensors."""
    def hp(x):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            return x.data_ptr()
        return x.ctypes.data
    st = appga_stats()
    _check(load_library().appga_reconstruct_host(ctx, mat, hp(g_host), hp(gamma_host),
                                                 hp(f_init_host), ctypes.byref(params),
                                                 hp(f_out_host), ctypes.byref(st),
                                                 _stream(stream)), "appga_reconstruct_host")
    return st


def appga_reconstruct_batched(ctx, mat, K, g, gamma, f_init, params, f_out, stream=None):
    """g, gamma: [K][m] device arrays; f_out: [K][d]; returns a list of K stats."""
    st = (appga_stats * K)()
    _check(load_library().appga_reconstruct_batched(ctx, mat, K, _ptr(g), _ptr(gamma),
                                                    _ptr(f_init), ctypes.byref(params), _ptr(f_out),
                                                    st, _stream(stream)),
           "appga_reconstruct_batched")
    return list(st)


def appga_gather_probe(ctx, mat, width: int = 64, launches: int = 20):
    """Rate (gathered GB/s) of the batched projectors' inner loop alone on
    this matrix, forward projection and back-projection (see appga.h):
    (fwd, bwd)."""
    fwd, bwd = ctypes.c_double(), ctypes.c_double()
    _check(load_library().appga_gather_probe(ctx, mat, width, launches, ctypes.byref(fwd),
                                             ctypes.byref(bwd)), "appga_gather_probe")
    return fwd.value, bwd.value


def appga_shoitv3d_grad(ctx, n_side, nz, f, lambda1, lambda2, eps, out, reg_out=None,
                        stream=None):
    """3-D SHOITV gradient of the slice-major volume f ([nz][n*n]) into out;
    reg_out (a device float64 scalar, optional) receives the regulariser."""
    _check(load_library().appga_shoitv3d_grad(ctx, n_side, nz, _ptr(f), lambda1, lambda2, eps,
                                              _ptr(out), _ptr(reg_out), _stream(stream)),
           "appga_shoitv3d_grad")


def appga_reconstruct_volume(ctx, mat, nz, g, gamma, f_init, params, f_out, stream=None):
    """APPGA on a volume of nz slices sharing the matrix: g, gamma [nz][m],
    f_init [nz][d] or None, f_out [nz][d] (device arrays).  Returns the
    volume's stats."""
    st = appga_stats()
    _check(load_library().appga_reconstruct_volume(ctx, mat, nz, _ptr(g), _ptr(gamma),
                                                   _ptr(f_init), ctypes.byref(params),
                                                   _ptr(f_out), ctypes.byref(st),
                                                   _stream(stream)),
           "appga_reconstruct_volume")
    return st


def appga_autotune_batched(ctx, mat, K, g, gamma, params) -> appga_batch_tuning:
    """Times launch schedules of the batched kernels on these K slices and
    keeps the best in the matrix handle (see appga.h)."""
    t = appga_batch_tuning()
    _check(load_library().appga_autotune_batched(ctx, mat, K, _ptr(g), _ptr(gamma),
                                                 ctypes.byref(params), ctypes.byref(t)),
           "appga_autotune_batched")
    return t


def appga_batch_schedule_get(mat, K: int, a_precision: int = 0) -> appga_batch_tuning:
    t = appga_batch_tuning(K=K, a_precision=a_precision)
    _check(load_library().appga_batch_schedule_get(mat, ctypes.byref(t)),
           "appga_batch_schedule_get")
    return t


def appga_batch_schedule_set(mat, tuning: appga_batch_tuning):
    _check(load_library().appga_batch_schedule_set(mat, ctypes.byref(tuning)),
           "appga_batch_schedule_set")


def appga_afppa_reconstruct(ctx, mat, g, gamma, f_init, params, f_out, b_out=None, c_out=None,
                            stream=None) -> appga_afppa_stats:
    """AFPPA for the non-smooth HOITV model (see appga.h); device buffers."""
    st = appga_afppa_stats()
    _check(load_library().appga_afppa_reconstruct(ctx, mat, _ptr(g), _ptr(gamma), _ptr(f_init),
                                                  ctypes.byref(params), _ptr(f_out), _ptr(b_out),
                                                  _ptr(c_out), ctypes.byref(st), _stream(stream)),
           "appga_afppa_reconstruct")
    return st


def appga_figures_of_merit(ctx, d, f, f_true, roi_h, roi_b, max_value, stream=None) -> appga_fom:
    """MSE, PSNR, RC and NRC of a device image against the ground truth
    (roi_h / roi_b: uint8 device masks, or None for both)."""
    out = appga_fom()
    _check(load_library().appga_figures_of_merit(ctx, d, _ptr(f), _ptr(f_true), _ptr(roi_h),
                                                 _ptr(roi_b), float(max_value), ctypes.byref(out),
                                                 _stream(stream)), "appga_figures_of_merit")
    return out


def appga_nofv(phi_k, phi_0, phi_ref) -> float:
    return load_library().appga_nofv(phi_k, phi_0, phi_ref)


def appga_central_line_profile(ctx, n_side, f, out, stream=None):
    _check(load_library().appga_central_line_profile(ctx, n_side, _ptr(f), _ptr(out),
                                                     _stream(stream)),
           "appga_central_line_profile")


def appga_objective_noalloc(ctx, mat, f, g, gamma, params, phi_out, stream=None):
    """Phi(f) into the device double phi_out[0]; allocates nothing (see appga.h)."""
    _check(load_library().appga_objective_noalloc(ctx, mat, _ptr(f), _ptr(g), _ptr(gamma),
                                                  ctypes.byref(params), _ptr(phi_out),
                                                  _stream(stream)), "appga_objective_noalloc")


def appga_validate_csr_host(m, d, row_ptr, col, val) -> int:
    import numpy as np
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    return load_library().appga_validate_csr_host(m, d, row_ptr.ctypes.data, col.ctypes.data,
                                                  val.ctypes.data)


def appga_kernel_times(ctx, mat, g, gamma, params, n_iters: int):
    """Mean device time (ms) of (pixel kernel, forward kernel) per launch."""
    tp, tf = ctypes.c_double(), ctypes.c_double()
    _check(load_library().appga_kernel_times(ctx, mat, _ptr(g), _ptr(gamma), ctypes.byref(params),
                                             n_iters, ctypes.byref(tp), ctypes.byref(tf)),
           "appga_kernel_times")
    return tp.value, tf.value


def _host_ptr(x) -> Optional[int]:
    """Address of a host buffer: a C-contiguous float32 numpy array or CPU tensor."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if x.is_cuda:
            raise ValueError("expected a host buffer")
        return x.data_ptr()
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous and x.dtype == np.float32):
        raise ValueError("host buffers must be C-contiguous float32 arrays")
    return x.ctypes.data


def appga_server_config_default() -> appga_server_config:
    c = appga_server_config()
    load_library().appga_server_config_default(ctypes.byref(c))
    return c


def server_config(**kw) -> appga_server_config:
    c = appga_server_config_default()
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(f"appga_server_config has no field {k!r}")
        setattr(c, k, v)
    return c


def appga_server_create(ctx, cfg: appga_server_config) -> int:
    h = _P()
    _check(load_library().appga_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)),
           "appga_server_create")
    return h.value


def appga_server_destroy(srv):
    _check(load_library().appga_server_destroy(srv), "appga_server_destroy")


def appga_server_add_geometry(srv, mat) -> int:
    gid = _I32()
    _check(load_library().appga_server_add_geometry(srv, mat, ctypes.byref(gid)),
           "appga_server_add_geometry")
    return gid.value


def appga_server_submit(srv, geometry, g_host, gamma_host, f_init_host, params) -> int:
    rid = _I64()
    _check(load_library().appga_server_submit(srv, geometry, _host_ptr(g_host),
                                              _host_ptr(gamma_host), _host_ptr(f_init_host),
                                              ctypes.byref(params), ctypes.byref(rid)),
           "appga_server_submit")
    return rid.value


def appga_server_step(srv) -> int:
    pending = _I32()
    _check(load_library().appga_server_step(srv, ctypes.byref(pending)), "appga_server_step")
    return pending.value


def appga_server_poll(srv, request) -> appga_request_stats:
    st = appga_request_stats()
    _check(load_library().appga_server_poll(srv, request, ctypes.byref(st)), "appga_server_poll")
    return st


def appga_server_collect(srv, request, f_out_host) -> appga_request_stats:
    st = appga_request_stats()
    _check(load_library().appga_server_collect(srv, request, _host_ptr(f_out_host),
                                               ctypes.byref(st)), "appga_server_collect")
    return st


def appga_server_get_summary(srv) -> appga_server_summary:
    s = appga_server_summary()
    _check(load_library().appga_server_get_summary(srv, ctypes.byref(s)),
           "appga_server_get_summary")
    return s


# ---- convenience objects ----

class Context:
    def __init__(self, device: int = 0):
        self.handle = appga_ctx_create(device)
        self.device = device

    def close(self):
        if self.handle:
            appga_ctx_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """Device copy of a system matrix (scipy CSR, FP32 values).

    bf16 also keeps a BF16 copy of the values; fold=False keeps the solver
    loop on the whole matrices even when A has the quarter-turn symmetry of a
    parallel-beam scanner (see appga_matrix_create)."""

    def __init__(self, ctx: Context, A, n_side: int, n_angles: int, bf16: bool = False,
                 fold: bool = True):
        self.ctx = ctx
        self.m, self.d = A.shape
        self.n_side = n_side
        self.n_angles = n_angles
        flags = (APPGA_A_BF16_COPY if bf16 else 0) | (0 if fold else APPGA_A_NO_FOLD)
        self.handle = appga_matrix_create(ctx.handle, self.m, self.d, n_side, n_angles, A.indptr,
                                          A.indices, A.data, flags)

    def info(self) -> appga_matrix_info:
        return appga_matrix_get_info(self.handle)

    def close(self):
        if self.handle:
            appga_matrix_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct(mat: Matrix, g, gamma, params: appga_params, f_init=None, stream=None):
    """Returns (f, stats) with f a new CUDA tensor."""
    import torch
    f_out = torch.empty(mat.d, dtype=torch.float32, device=g.device)
    st = appga_reconstruct(mat.ctx.handle, mat.handle, g, gamma, f_init, params, f_out, stream)
    return f_out, st


def nan() -> float:
    return math.nan


class Server:
    """Continuous-batching server (appga_server.h) over registered matrices."""

    def __init__(self, ctx: Context, **cfg):
        self.ctx = ctx
        self.handle = appga_server_create(ctx.handle, server_config(**cfg))
        self.geometries = []
        self._geom_of = {}

    def add_geometry(self, mat: Matrix) -> int:
        gid = appga_server_add_geometry(self.handle, mat.handle)
        self.geometries.append(mat)
        return gid

    def submit(self, geometry: int, g, gamma, params: appga_params, f_init=None) -> int:
        rid = appga_server_submit(self.handle, geometry, g, gamma, f_init, params)
        self._geom_of[rid] = geometry
        return rid

    def step(self) -> int:
        return appga_server_step(self.handle)

    def poll(self, request: int) -> appga_request_stats:
        return appga_server_poll(self.handle, request)

    def collect(self, request: int):
        """(image as a float32 numpy array, stats) of a finished request."""
        import numpy as np
        f = np.empty(self.geometries[self._geom_of[request]].d, np.float32)
        st = appga_server_collect(self.handle, request, f)
        del self._geom_of[request]
        return f, st

    def summary(self) -> appga_server_summary:
        return appga_server_get_summary(self.handle)

    def close(self):
        if self.handle:
            appga_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
