"""ctypes declarations of include/reallife.h and the library loader (no fallback)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# REALLIFE_DEBUG=1 loads the bounds-checked debug build (libreallife_debug.so) instead
DEBUG = os.environ.get("REALLIFE_DEBUG", "0") not in ("", "0")
_LIB_PATH = os.path.join(_HERE, "libreallife_debug.so" if DEBUG else "libreallife.so")
_lock = threading.Lock()
_lib = None

# every symbol the header declares
EXPORTS = [
    "reallife_workspace_bytes", "reallife_render", "reallife_hsgd_step", "reallife_refine",
    "reallife_downsample_f32", "reallife_select", "reallife_select_keys", "reallife_loss_grad",
    "reallife_sparse_update", "reallife_render_backward", "reallife_warp_offsets", "reallife_trace_enable",
    "reallife_trace_read", "reallife_strerror", "reallife_last_error", "reallife_set_kernel_path",
    "reallife_device_status", "reallife_hsgd_step_noalloc", "reallife_trace_release_captured",
    "reallife_gradient_volume_workspace_bytes", "reallife_gradient_volume", "reallife_lgd_net_bytes",
    "reallife_lgd_prepare", "reallife_lgd_workspace_bytes", "reallife_lgd_forward",
    "reallife_lgd_step_workspace_bytes", "reallife_lgd_step", "reallife_selftest_wait_timeout",
    "reallife_batch_table_bytes", "reallife_batch_prepare", "reallife_hsgd_step_batch",
    "reallife_selftest_bounds", "reallife_debug_build",
    "reallife_metrics_workspace_bytes", "reallife_image_metrics", "reallife_kept_mass",
]


class RealLifeError(RuntimeError):
    pass


class RlCamera(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class RlMpi(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int), ("near_", ctypes.c_double),
                ("far_", ctypes.c_double), ("dtype", ctypes.c_int), ("data", ctypes.c_void_p), ("ref", RlCamera)]


class RlHsgdParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("lambda_", ctypes.c_float), ("clamp01", ctypes.c_int), ("level", ctypes.c_int),
                ("selection", ctypes.c_int), ("lambda_s", ctypes.c_float)]


class RlBatchItem(ctypes.Structure):
    _fields_ = [("mpi", ctypes.POINTER(RlMpi)), ("images", ctypes.c_void_p), ("src", ctypes.POINTER(RlCamera)),
                ("N", ctypes.c_int), ("params", RlHsgdParams), ("loss_out", ctypes.c_void_p), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t)]


class RlLgdParams(ctypes.Structure):
    _fields_ = [("c_in", ctypes.c_int), ("eps", ctypes.c_float),
                ("conv_w", ctypes.c_void_p * 5), ("conv_b", ctypes.c_void_p * 5),
                ("bn_gamma", ctypes.c_void_p * 5), ("bn_beta", ctypes.c_void_p * 5),
                ("bn_mean", ctypes.c_void_p * 5), ("bn_var", ctypes.c_void_p * 5),
                ("out_w", ctypes.c_void_p), ("out_b", ctypes.c_void_p)]


class RlTraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


def camera(c) -> RlCamera:
    """Host camera struct from an object with K, R, t (or a (K, R, t) tuple)."""
    K, R, t = (c.K, c.R, c.t) if hasattr(c, "K") else c
    s = RlCamera()
    s.K[:] = np.asarray(K, dtype=np.float64).reshape(9).tolist()
    s.R[:] = np.asarray(R, dtype=np.float64).reshape(9).tolist()
    s.t[:] = np.asarray(t, dtype=np.float64).reshape(3).tolist()
    return s


def cameras(cs):
    arr = (RlCamera * len(cs))()
    for i, c in enumerate(cs):
        arr[i] = camera(c)
    return arr


def path() -> str:
    return _LIB_PATH


def _declare(lib):
    c_int, c_float, c_size_t, vp = ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
    mpi_p, cam_p, par_p = ctypes.POINTER(RlMpi), ctypes.POINTER(RlCamera), ctypes.POINTER(RlHsgdParams)
    sig = {
        "reallife_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
        "reallife_render": (c_int, [mpi_p, cam_p, c_int, vp, vp]),
        "reallife_hsgd_step": (c_int, [mpi_p, vp, cam_p, c_int, par_p, vp, vp, vp, c_size_t, vp]),
        "reallife_hsgd_step_noalloc": (c_int, [mpi_p, vp, cam_p, c_int, par_p, vp, vp, vp]),
        "reallife_refine": (c_int, [mpi_p, vp, cam_p, c_int, par_p, ctypes.POINTER(c_int), c_int, vp, vp, c_size_t,
                                    vp]),
        "reallife_downsample_f32": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, vp, vp]),
        "reallife_select": (c_int, [mpi_p, c_int, c_int, vp, vp, vp]),
        "reallife_select_keys": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, vp, vp, vp]),
        "reallife_loss_grad": (c_int, [mpi_p, vp, cam_p, c_int, vp, c_int, vp, vp, vp, c_size_t, vp]),
        "reallife_sparse_update": (c_int, [mpi_p, vp, vp, c_int, c_int, c_float, c_int, vp]),
        "reallife_render_backward": (c_int, [mpi_p, cam_p, c_int, vp, vp, vp]),
        "reallife_warp_offsets": (c_int, [mpi_p, cam_p, vp, vp]),
        "reallife_trace_enable": (c_int, [c_int]),
        "reallife_trace_release_captured": (c_int, []),
        "reallife_trace_read": (c_int, [ctypes.POINTER(RlTraceEntry), c_int, ctypes.POINTER(c_int)]),
        "reallife_strerror": (ctypes.c_char_p, [c_int]),
        "reallife_set_kernel_path": (c_int, [c_int]),
        "reallife_device_status": (c_int, [c_int, ctypes.POINTER(ctypes.c_uint)]),
        "reallife_selftest_wait_timeout": (c_int, [ctypes.c_uint, vp]),
        "reallife_selftest_bounds": (c_int, [vp]),
        "reallife_metrics_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
        "reallife_image_metrics": (c_int, [vp, vp, c_int, c_int, c_int, vp, vp, c_size_t, vp]),
        "reallife_kept_mass": (c_int, [mpi_p, vp, vp, vp, c_size_t, vp]),
        "reallife_debug_build": (c_int, []),
        "reallife_last_error": (ctypes.c_char_p, []),
        "reallife_gradient_volume_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
        "reallife_gradient_volume": (c_int, [mpi_p, vp, cam_p, c_int, c_int, c_int, c_int, vp, vp, vp, c_size_t,
                                             vp]),
        "reallife_batch_table_bytes": (c_size_t, [c_int]),
        "reallife_batch_prepare": (c_int, [ctypes.POINTER(RlBatchItem), c_int, vp, c_size_t]),
        "reallife_hsgd_step_batch": (c_int, [vp, vp, c_size_t, vp]),
        "reallife_lgd_net_bytes": (c_size_t, []),
        "reallife_lgd_prepare": (c_int, [ctypes.POINTER(RlLgdParams), vp, vp]),
        "reallife_lgd_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
        "reallife_lgd_forward": (c_int, [vp, vp, c_int, c_int, c_int, c_int, vp, vp, c_size_t, vp]),
        "reallife_lgd_step_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
        "reallife_lgd_step": (c_int, [mpi_p, vp, cam_p, c_int, c_int, c_int, c_int, c_int, vp, vp, vp, c_size_t, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """The loaded library; builds it in-tree with nvcc when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            try:
                p = _build.build(debug=DEBUG)
            except Exception as e:  # no silent fallback: the CUDA library is the product
                raise RealLifeError(f"libreallife is not available and could not be built: {e}") from e
            l = ctypes.CDLL(p)
            _declare(l)
            _lib = l
    return _lib


def check(fn: str, status: int):
    if status != 0:
        l = lib()
        raise RealLifeError(f"{fn}: {l.reallife_strerror(status).decode()} ({l.reallife_last_error().decode()})")
