"""B300-native chunked 3D volume filtering (Gaussian, derivative-of-Gaussian
features, grayscale morphology) behind the libhp C ABI.

The package loads the in-tree libhp.so (built by ``build.py``) and raises
ImportError when it is missing; no operation has a fallback.
"""
from .api import (G, GM, LOG, HPError, close3d, dilate3d, erode3d, filterbank3d,
                  filterbank3d_adjoint, gaussian3d, get_devices, get_memory_budget, hessian3d,
                  morph3d_backward, multi3d, open3d, plan_bricks, probe_fp32_fma, release_cache,
                  selftest_wait_timeout,
                  set_brick_shard, set_devices, set_memory_budget, shard_bricks, stats,
                  stream_status, threshold3d, threshold_box3d, threshold_local3d, tophat3d,
                  unsharp3d, version)
from ._lib import (HP_DEVICE, HP_F16, HP_F32, HP_HOST, HP_SE_BALL, HP_SE_CUBE, HP_U8, HP_U16,
                   EXPORTS, LIB_PATH)

__all__ = [
    "G", "GM", "LOG", "HPError", "close3d", "dilate3d", "erode3d", "filterbank3d",
    "filterbank3d_adjoint", "gaussian3d", "get_devices", "get_memory_budget", "hessian3d",
    "morph3d_backward", "multi3d", "threshold_box3d",
    "open3d", "plan_bricks", "probe_fp32_fma", "release_cache", "selftest_wait_timeout", "set_brick_shard",
    "set_devices", "set_memory_budget", "shard_bricks", "stats", "stream_status", "threshold3d",
    "threshold_local3d", "tophat3d", "unsharp3d", "version", "HP_DEVICE", "HP_F16", "HP_F32",
    "HP_HOST", "HP_SE_BALL", "HP_SE_CUBE", "HP_U8", "HP_U16", "EXPORTS", "LIB_PATH",
]
