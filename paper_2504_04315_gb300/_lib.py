"""ctypes view of the C ABI declared in include/npm.h.

Loading fails loudly (RuntimeError) when the CUDA library has not been
built: there is no CPU fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB

MAX_LEVELS = 32
MAX_LAYERS = 8
FRAME_BOUNCE_STATS = 16

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NUMERIC, \
    ERR_UNSUPPORTED, ERR_IO = range(9)
STATUS_NAMES = ["NPM_OK", "NPM_ERR_INVALID_ARG", "NPM_ERR_OOM", "NPM_ERR_CUDA",
                "NPM_ERR_CAPACITY", "NPM_ERR_TIMEOUT", "NPM_ERR_NUMERIC",
                "NPM_ERR_UNSUPPORTED", "NPM_ERR_IO"]


class NpmConfig(C.Structure):
    _fields_ = [
        ("mode", C.c_int), ("n_levels", C.c_int), ("feat_per_level", C.c_int),
        ("log2_table", C.c_int), ("level_res", C.c_int * MAX_LEVELS),
        ("n_layers", C.c_int), ("widths", C.c_int * (MAX_LAYERS + 1)), ("K", C.c_int),
        ("kappa_act", C.c_int), ("precision", C.c_int),
        ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
        ("max_batch", C.c_int64), ("seed", C.c_uint64),
    ]


class NpmServerStats(C.Structure):
    _fields_ = [
        ("batches", C.c_int64), ("requests_done", C.c_int64), ("queries_done", C.c_int64),
        ("train_done", C.c_int64), ("max_requests_per_batch", C.c_int64),
        ("pool_queries", C.c_int64), ("pool_peak_used", C.c_int64),
        ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double),
    ]


class NpmFrameConfig(C.Structure):
    _fields_ = [
        ("paths", C.c_int64), ("bounces", C.c_int), ("survival", C.c_float),
        ("train_batch", C.c_int64), ("uniform_frac", C.c_float), ("seed", C.c_uint64),
        ("use_graph", C.c_int), ("max_frames", C.c_int),
    ]


class NpmFrameStats(C.Structure):
    _fields_ = [
        ("frames", C.c_int64), ("queries", C.c_int64), ("seconds", C.c_double),
        ("queries_per_s", C.c_double), ("bounce_p50_ms", C.c_double),
        ("bounce_p99_ms", C.c_double), ("frame_ms_mean", C.c_double),
        ("train_ms_mean", C.c_double), ("last_loss", C.c_float),
        ("query_ms_mean", C.c_double), ("advance_ms_mean", C.c_double),
        ("bounce_queries", C.c_double * FRAME_BOUNCE_STATS),
        ("bounce_query_ms", C.c_double * FRAME_BOUNCE_STATS),
    ]


class NpmUnitPeaks(C.Structure):
    _fields_ = [
        ("fp32_fma_tflops", C.c_double), ("fp32_fma_scalar_tflops", C.c_double),
        ("mufu_gops", C.c_double),
        ("l2_sector_read_gbs", C.c_double), ("l2_atomic_gops", C.c_double),
        ("l2_atomic_v2_gops", C.c_double), ("l2_atomic_v4_gops", C.c_double), ("sm_count", C.c_int),
        ("max_sm_clock_mhz", C.c_double),
    ]


vp = C.c_void_p
i64 = C.c_int64
f32 = C.c_float
st = C.c_int

# name -> (restype, argtypes); every symbol include/npm.h declares.
SIGNATURES = {
    "npm_create": (st, [C.POINTER(NpmConfig), C.POINTER(vp)]),
    "npm_destroy": (st, [vp]),
    "npm_query_sample": (st, [vp, i64, vp, vp, vp, i64, f32, vp, vp, vp, vp]),
    "npm_query_sample_host": (st, [vp, i64, vp, vp, vp, i64, f32, vp, vp, vp]),
    "npm_eval_pdf": (st, [vp, i64, vp, vp, vp, i64, vp, vp]),
    "npm_eval_log_pdf": (st, [vp, i64, vp, vp, vp, i64, vp, vp]),
    "npm_debug_bounds_violations": (i64, []),
    "npm_train_step": (st, [vp, i64, vp, vp, vp, vp, vp, i64, vp, vp]),
    "npm_backward": (st, [vp, i64, vp, vp, vp, vp, i64, vp]),
    "npm_adam_step": (st, [vp, vp]),
    "npm_num_params": (i64, [vp]),
    "npm_set_params": (st, [vp, vp, i64]),
    "npm_get_params": (st, [vp, vp, i64]),
    "npm_get_grads": (st, [vp, vp, i64]),
    "npm_set_params_device": (st, [vp, vp, i64, vp]),
    "npm_get_grads_device": (st, [vp, vp, i64, vp]),
    "npm_params_device": (vp, [vp]),
    "npm_grads_device": (vp, [vp]),
    "npm_set_ema": (st, [vp, f32, vp]),
    "npm_get_ema_params": (st, [vp, vp, i64]),
    "npm_get_adam": (st, [vp, C.POINTER(C.c_int), vp, vp]),
    "npm_set_adam": (st, [vp, C.c_int, vp, vp]),
    "npm_grid_indices": (st, [vp, i64, vp, i64, vp, vp]),
    "npm_save": (st, [vp, C.c_char_p]),
    "npm_load": (st, [vp, C.c_char_p]),
    "npm_check_device_status": (st, [vp, vp]),
    "npm_set_wait_limit": (st, [vp, i64]),
    "npm_pdf_integral": (st, [vp, i64, vp, vp, i64, i64, vp, vp, vp, vp]),
    "npm_last_error": (C.c_char_p, []),
    "npm_wavefront_create": (st, [vp, C.POINTER(NpmFrameConfig), C.POINTER(vp)]),
    "npm_wavefront_run": (st, [vp, C.c_int, vp, C.POINTER(NpmFrameStats)]),
    "npm_wavefront_destroy": (st, [vp]),
    "npm_scene_generate": (st, [C.c_uint64, i64, C.c_int, vp, vp, vp, C.c_int, i64, vp]),
    "npm_scene_radiance": (st, [C.c_int, C.c_uint64, i64, vp, vp, vp, i64, vp, vp, vp]),
    "npm_server_create": (st, [vp, i64, C.POINTER(vp)]),
    "npm_server_submit_query": (st, [vp, i64, vp, vp, vp, i64, f32, vp, vp, C.POINTER(C.c_uint64)]),
    "npm_server_submit_train": (st, [vp, i64, vp, vp, vp, vp, vp, i64, C.POINTER(C.c_uint64)]),
    "npm_server_hold": (st, [vp, C.c_int]),
    "npm_server_wait": (st, [vp, C.c_uint64, C.POINTER(C.c_double)]),
    "npm_server_get_stats": (st, [vp, C.POINTER(NpmServerStats)]),
    "npm_server_destroy": (st, [vp]),
    "npm_eval_pdf_noalloc": (st, [C.POINTER(NpmConfig), vp, i64, vp, vp, vp, i64, vp, vp]),
    "npm_measure_unit_peaks": (st, [C.POINTER(NpmUnitPeaks), vp]),
}

_lib = None


def load():
    """The loaded library (ctypes.CDLL) with typed entry points."""
    global _lib
    if _lib is not None:
        return _lib
    # NPM_LIBRARY selects another in-tree build (the bounds-checking debug
    # build of _build.build_debug()).
    path = os.environ.get("NPM_LIBRARY") or LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is not built; run paper_2504_04315_gb300._build.build() "
            "(or __graft_entry__.build()). There is no CPU fallback.")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NpmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().npm_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != OK:
        raise NpmError(status, where)
