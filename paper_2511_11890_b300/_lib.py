"""ctypes binding to libhp.so, the C ABI declared in include/hp.h.

Argument marshalling only: every step of the filtering path runs in the
library's CUDA kernels. Importing this module loads the in-tree libhp.so and
raises ImportError when it is missing; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhp.so")

HP_OK, HP_ERR_INVALID_ARG, HP_ERR_UNSUPPORTED, HP_ERR_BUDGET = 0, 1, 2, 3
HP_ERR_OOM, HP_ERR_CUDA, HP_ERR_TIMEOUT, HP_ERR_INTERNAL = 4, 5, 6, 7
STATUS_NAMES = {0: "HP_OK", 1: "HP_ERR_INVALID_ARG", 2: "HP_ERR_UNSUPPORTED", 3: "HP_ERR_BUDGET",
                4: "HP_ERR_OOM", 5: "HP_ERR_CUDA", 6: "HP_ERR_TIMEOUT", 7: "HP_ERR_INTERNAL"}
HP_U8, HP_U16, HP_F16, HP_F32 = 0, 1, 2, 3
HP_HOST, HP_DEVICE = 0, 1
HP_SE_CUBE, HP_SE_BALL = 0, 1
HP_FILTER_G, HP_FILTER_GM, HP_FILTER_LOG = 0, 1, 2
HP_LOCAL_MEAN, HP_LOCAL_NIBLACK, HP_LOCAL_SAUVOLA = 0, 1, 2
HP_HESSIAN_COMPONENTS, HP_HESSIAN_EIGENVALUES = 0, 1

# Every entry point declared in include/hp.h.
EXPORTS = [
    "hp_volume_create", "hp_volume_destroy", "hp_set_memory_budget", "hp_get_memory_budget",
    "hp_gaussian3d", "hp_filterbank3d", "hp_filterbank3d_bricks", "hp_erode3d", "hp_dilate3d",
    "hp_open3d", "hp_close3d", "hp_tophat3d", "hp_unsharp3d", "hp_threshold_local3d",
    "hp_threshold3d", "hp_threshold_box3d", "hp_hessian3d", "hp_multi3d", "hp_filterbank3d_adjoint",
    "hp_morph3d_backward",
    "hp_morph3d_backward_noalloc", "hp_set_devices", "hp_get_devices", "hp_set_brick_shard",
    "hp_plan_bricks",
    "hp_stream_status", "hp_selftest_wait_timeout", "hp_probe_fp32_fma", "hp_release_cache", "hp_get_stats", "hp_last_error", "hp_version",
]


class HPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class hp_filter(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double)]


class hp_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double), ("order", ctypes.c_int * 3),
                ("se", ctypes.c_int), ("radius", ctypes.c_int)]


HP_OP_GAUSSIAN, HP_OP_ERODE, HP_OP_DILATE = 0, 1, 2


class hp_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3)]


class hp_stats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("peak_device_bytes", ctypes.c_size_t),
                ("live_device_bytes", ctypes.c_size_t), ("cached_device_bytes", ctypes.c_size_t),
                ("pinned_host_bytes", ctypes.c_size_t), ("bricks", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("wall_ms", ctypes.c_double), ("bank_kernels", ctypes.c_uint64)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhp.so not built ({LIB_PATH}); run "
                          "`python paper_2511_11890_b300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i, d, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hp_volume_create": [pvp, vp, i, i, i64, i64, i64],
        "hp_volume_destroy": [vp],
        "hp_set_memory_budget": [sz],
        "hp_get_memory_budget": [ctypes.POINTER(sz)],
        "hp_gaussian3d": [vp, vp, d, d, ctypes.POINTER(ctypes.c_int), vp],
        "hp_filterbank3d": [vp, pvp, ctypes.POINTER(hp_filter), i, vp],
        "hp_filterbank3d_bricks": [vp, pvp, ctypes.POINTER(hp_filter), i, ctypes.POINTER(hp_box), i, vp],
        "hp_erode3d": [vp, vp, i, i, vp],
        "hp_dilate3d": [vp, vp, i, i, vp],
        "hp_open3d": [vp, vp, i, i, vp],
        "hp_close3d": [vp, vp, i, i, vp],
        "hp_tophat3d": [vp, vp, i, i, vp],
        "hp_unsharp3d": [vp, vp, d, d, vp],
        "hp_threshold_local3d": [vp, vp, d, d, vp],
        "hp_threshold3d": [vp, vp, d, vp],
        "hp_threshold_box3d": [vp, vp, i, i, d, d, vp],
        "hp_hessian3d": [vp, pvp, i, d, vp],
        "hp_multi3d": [vp, pvp, ctypes.POINTER(hp_op), i, vp],
        "hp_filterbank3d_adjoint": [vp, pvp, ctypes.POINTER(hp_filter), i, vp, vp],
        "hp_morph3d_backward": [vp, vp, i, i, i, vp, i, vp],
        "hp_morph3d_backward_noalloc": [vp, vp, i, i, i, vp, i, vp],
        "hp_set_devices": [ctypes.POINTER(i), i],
        "hp_get_devices": [ctypes.POINTER(i), i, ctypes.POINTER(i)],
        "hp_set_brick_shard": [i, i],
        "hp_plan_bricks": [i64, i64, i64, i, sz, sz, sz, i, i, ctypes.POINTER(hp_box),
                           ctypes.POINTER(hp_box), i, ctypes.POINTER(i)],
        "hp_stream_status": [vp],
        "hp_selftest_wait_timeout": [vp],
        "hp_probe_fp32_fma": [vp, i, ctypes.POINTER(d)],
        "hp_release_cache": [],
        "hp_get_stats": [ctypes.POINTER(hp_stats)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.hp_last_error.restype = ctypes.c_char_p
    lib.hp_last_error.argtypes = []
    lib.hp_version.restype = ctypes.c_char_p
    lib.hp_version.argtypes = []
    return lib


lib = _load()


def check(status: int):
    if status != HP_OK:
        raise HPError(status, lib.hp_last_error().decode(errors="replace"))
