"""Python front end of libhp: one function per C entry point.

Each function takes torch tensors (CUDA -> device mode, asynchronous on the
current stream; CPU -> out-of-core host mode) or numpy arrays (host mode),
shape (nz, ny, nx), C-contiguous, and passes raw pointers and sizes through
the C ABI. It allocates outputs when none are given and does nothing else:
all arithmetic runs in libhp's kernels.
"""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (HP_DEVICE, HP_F16, HP_F32, HP_HOST, HP_SE_BALL, HP_SE_CUBE, HP_U8, HP_U16,
                   HPError, check, hp_box, hp_filter, hp_stats, lib)

G, GM, LOG = _lib.HP_FILTER_G, _lib.HP_FILTER_GM, _lib.HP_FILTER_LOG
SE = {"cube": HP_SE_CUBE, "ball": HP_SE_BALL, HP_SE_CUBE: HP_SE_CUBE, HP_SE_BALL: HP_SE_BALL}

_TORCH_DT = {torch.uint8: HP_U8, torch.uint16: HP_U16, torch.float16: HP_F16,
             torch.float32: HP_F32}
_NP_DT = {np.dtype(np.uint8): HP_U8, np.dtype(np.uint16): HP_U16, np.dtype(np.float16): HP_F16,
          np.dtype(np.float32): HP_F32}
_HP_TO_TORCH = {v: k for k, v in _TORCH_DT.items()}
_HP_TO_NP = {v: k for k, v in _NP_DT.items()}


def _dtype_code(a) -> int:
    if isinstance(a, torch.Tensor):
        if a.dtype not in _TORCH_DT:
            raise TypeError(f"unsupported dtype {a.dtype}")
        return _TORCH_DT[a.dtype]
    if a.dtype not in _NP_DT:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return _NP_DT[a.dtype]


class _View:
    """A non-owning hp_volume over a tensor or array, destroyed on exit."""

    def __init__(self, a):
        if a.ndim != 3:
            raise ValueError("volumes are 3D arrays (nz, ny, nx)")
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            ptr, loc = a.data_ptr(), (HP_DEVICE if a.is_cuda else HP_HOST)
        else:
            if not a.flags.c_contiguous:
                raise ValueError("array must be C-contiguous")
            ptr, loc = a.ctypes.data, HP_HOST
        self.loc = loc
        self.h = ctypes.c_void_p()
        nz, ny, nx = a.shape
        check(lib.hp_volume_create(ctypes.byref(self.h), ctypes.c_void_p(ptr), _dtype_code(a), loc,
                                   nx, ny, nz))

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        lib.hp_volume_destroy(self.h)


def _empty_like(x, dtype_code: int):
    if isinstance(x, torch.Tensor):
        return torch.empty(x.shape, dtype=_HP_TO_TORCH[dtype_code], device=x.device,
                           pin_memory=bool(not x.is_cuda and x.is_pinned()))
    return np.empty(x.shape, _HP_TO_NP[dtype_code])


def _ctx(x):
    if isinstance(x, torch.Tensor) and x.is_cuda:
        return torch.cuda.device(x.device)
    return contextlib.nullcontext()


def _stream(x, stream):
    if isinstance(x, torch.Tensor) and x.is_cuda:
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(0)


def gaussian3d(x, sigma: float, order=(0, 0, 0), truncate: float = 3.0, out=None,
               out_dtype: int = HP_F32, stream=None):
    """Separable Gaussian / derivative filter; order = (oz, oy, ox)."""
    if out is None:
        out = _empty_like(x, out_dtype)
    ordv = (ctypes.c_int * 3)(*[int(o) for o in order])
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_gaussian3d(vi, vo, float(sigma), float(truncate), ordv, _stream(x, stream)))
    return out


def erode3d(x, se="ball", radius: int = 1, out=None, stream=None):
    if out is None:
        out = _empty_like(x, _dtype_code(x))
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_erode3d(vi, vo, SE[se], int(radius), _stream(x, stream)))
    return out


def dilate3d(x, se="ball", radius: int = 1, out=None, stream=None):
    if out is None:
        out = _empty_like(x, _dtype_code(x))
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_dilate3d(vi, vo, SE[se], int(radius), _stream(x, stream)))
    return out


def _compose(fn, x, se, radius, out, stream):
    if out is None:
        out = _empty_like(x, _dtype_code(x))
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(fn(vi, vo, SE[se], int(radius), _stream(x, stream)))
    return out


def open3d(x, se="ball", radius: int = 1, out=None, stream=None):
    """Opening (erosion, then dilation); device tensors only."""
    return _compose(lib.hp_open3d, x, se, radius, out, stream)


def close3d(x, se="ball", radius: int = 1, out=None, stream=None):
    """Closing (dilation, then erosion); device tensors only."""
    return _compose(lib.hp_close3d, x, se, radius, out, stream)


def tophat3d(x, se="ball", radius: int = 1, out=None, stream=None):
    """White top-hat, x - opening(x); device tensors only."""
    return _compose(lib.hp_tophat3d, x, se, radius, out, stream)


def unsharp3d(x, sigma: float, amount: float = 1.0, out=None, stream=None):
    """Unsharp mask x + amount * (x - G_sigma x) as float32; device tensors only."""
    if out is None:
        out = _empty_like(x, HP_F32)
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_unsharp3d(vi, vo, float(sigma), float(amount), _stream(x, stream)))
    return out


def threshold_local3d(x, sigma: float, offset: float = 0.0, out=None, stream=None):
    """Gaussian local threshold x > G_sigma x - offset as uint8; device tensors only."""
    if out is None:
        out = _empty_like(x, HP_U8)
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_threshold_local3d(vi, vo, float(sigma), float(offset), _stream(x, stream)))
    return out


def threshold3d(x, t: float = 0.5, out=None, stream=None):
    if out is None:
        out = _empty_like(x, HP_U8)
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_threshold3d(vi, vo, float(t), _stream(x, stream)))
    return out


LOCAL = {"mean": _lib.HP_LOCAL_MEAN, "niblack": _lib.HP_LOCAL_NIBLACK,
         "sauvola": _lib.HP_LOCAL_SAUVOLA}


def threshold_box3d(x, method="niblack", radius: int = 7, k: float = 0.2, c: float = 0.0,
                    out=None, stream=None):
    """Box-window local threshold: u8 = x > T, T from the window mean m and
    standard deviation s: 'mean' m - c, 'niblack' m + k s, 'sauvola'
    m (1 + k (s / c - 1)) (c = R)."""
    if out is None:
        out = _empty_like(x, HP_U8)
    with _ctx(x), _View(x) as vi, _View(out) as vo:
        check(lib.hp_threshold_box3d(vi, vo, int(LOCAL.get(method, method)), int(radius), float(k),
                                     float(c), _stream(x, stream)))
    return out


def hessian3d(x, sigma: float, eigenvalues: bool = False, outs=None, out_dtype: int = HP_F32,
              stream=None):
    """Hessian features: the six components (Dzz, Dyy, Dxx, Dzy, Dzx, Dyx),
    or with eigenvalues=True the three ascending eigenvalues per voxel."""
    n = 3 if eigenvalues else 6
    if outs is None:
        outs = [_empty_like(x, out_dtype) for _ in range(n)]
    views = [_View(o) for o in outs]
    try:
        handles = (ctypes.c_void_p * len(outs))(*[v.h.value for v in views])
        what = _lib.HP_HESSIAN_EIGENVALUES if eigenvalues else _lib.HP_HESSIAN_COMPONENTS
        with _ctx(x), _View(x) as vi:
            check(lib.hp_hessian3d(vi, handles, what, float(sigma), _stream(x, stream)))
    finally:
        for v in views:
            v.__exit__()
    return outs


def multi3d(x, ops, outs=None, stream=None):
    """Several filters of x in one pass: ops is a list of
    ("gauss", sigma[, (oz, oy, ox)][, out_dtype]) and ("erode" | "dilate",
    se, radius); outputs default to float32 (Gaussians) and x's dtype
    (morphology). Host inputs stream through the device once for all ops."""
    arr = (_lib.hp_op * len(ops))()
    made = []
    for i, q in enumerate(ops):
        kind = q[0]
        if kind == "gauss":
            arr[i].kind = _lib.HP_OP_GAUSSIAN
            arr[i].sigma = float(q[1])
            order = q[2] if len(q) > 2 else (0, 0, 0)
            for a in range(3):
                arr[i].order[a] = int(order[a])
            made.append(q[3] if len(q) > 3 else HP_F32)
        elif kind in ("erode", "dilate"):
            arr[i].kind = _lib.HP_OP_ERODE if kind == "erode" else _lib.HP_OP_DILATE
            arr[i].se = SE[q[1]]
            arr[i].radius = int(q[2])
            made.append(_dtype_code(x))
        else:
            raise ValueError(f"unknown op {kind!r}")
    if outs is None:
        outs = [_empty_like(x, dt) for dt in made]
    views = [_View(o) for o in outs]
    try:
        handles = (ctypes.c_void_p * len(outs))(*[v.h.value for v in views])
        with _ctx(x), _View(x) as vi:
            check(lib.hp_multi3d(vi, handles, arr, len(ops), _stream(x, stream)))
    finally:
        for v in views:
            v.__exit__()
    return outs


def _filters(filters):
    arr = (hp_filter * len(filters))()
    for i, (k, s) in enumerate(filters):
        arr[i].kind = int(k)
        arr[i].sigma = float(s)
    return arr


def _boxes(bricks):
    bricks = np.asarray(bricks, np.int64).reshape(-1, 6)
    arr = (hp_box * len(bricks))()
    for i, b in enumerate(bricks):
        for a in range(3):
            arr[i].lo[a] = int(b[a])
            arr[i].hi[a] = int(b[3 + a])
    return arr


def filterbank3d(x, filters, outs=None, out_dtype: int = HP_F16, bricks=None, stream=None):
    """Outputs of filters [(kind, sigma), ...] in one persistent launch."""
    if outs is None:
        outs = [_empty_like(x, out_dtype) for _ in filters]
    views = [_View(o) for o in outs]
    try:
        handles = (ctypes.c_void_p * len(outs))(*[v.h.value for v in views])
        with _ctx(x), _View(x) as vi:
            if bricks is None:
                check(lib.hp_filterbank3d(vi, handles, _filters(filters), len(filters),
                                          _stream(x, stream)))
            else:
                bx = _boxes(bricks)
                check(lib.hp_filterbank3d_bricks(vi, handles, _filters(filters), len(filters), bx,
                                                 len(bx), _stream(x, stream)))
    finally:
        for v in views:
            v.__exit__()
    return outs


def filterbank3d_adjoint(x, gouts, filters, gin=None, stream=None):
    """gin = sum_i J_i^T gouts[i] (device, float32)."""
    if gin is None:
        gin = _empty_like(x, HP_F32)
    views = [_View(g) for g in gouts]
    try:
        handles = (ctypes.c_void_p * len(gouts))(*[v.h.value for v in views])
        with _ctx(x), _View(x) as vi, _View(gin) as vg:
            check(lib.hp_filterbank3d_adjoint(vi, handles, _filters(filters), len(filters), vg,
                                              _stream(x, stream)))
    finally:
        for v in views:
            v.__exit__()
    return gin


def morph3d_backward(x, gout, dilate: bool, se="cube", radius: int = 1, gin=None,
                     accumulate: bool = False, stream=None):
    """Subgradient of erosion / dilation (ties to the smallest source index)."""
    if gin is None:
        gin = _empty_like(x, HP_F32)
        accumulate = False
    with _ctx(x), _View(x) as vi, _View(gout) as vg, _View(gin) as vo:
        check(lib.hp_morph3d_backward(vi, vg, int(bool(dilate)), SE[se], int(radius), vo,
                                      int(bool(accumulate)), _stream(x, stream)))
    return gin


def plan_bricks(shape, halo: int, in_bytes: int, out_bytes: int, budget: int, stages: int = 3,
                min_bricks: int = 8):
    """Host-only chunk plan: (cores, in_boxes) as (n, 6) arrays [z0,y0,x0,z1,y1,x1]."""
    nz, ny, nx = shape
    n = ctypes.c_int(0)
    check(lib.hp_plan_bricks(nx, ny, nz, halo, in_bytes, out_bytes, budget, stages, min_bricks,
                             None, None, 0, ctypes.byref(n)))
    cores = (hp_box * n.value)()
    boxes = (hp_box * n.value)()
    check(lib.hp_plan_bricks(nx, ny, nz, halo, in_bytes, out_bytes, budget, stages, min_bricks,
                             cores, boxes, n.value, ctypes.byref(n)))
    to_np = lambda arr: np.array([[*b.lo, *b.hi] for b in arr], np.int64).reshape(-1, 6)
    return to_np(cores), to_np(boxes)


def shard_bricks(n: int, rank: int, world: int):
    """Indices of the bricks rank `rank` of `world` processes: round-robin over
    the plan (brick i goes to rank i mod world), as the paper's multi-GPU
    chunk scheduling does (Sec. III-D). Bricks are independent given their
    read-only halos, so ranks exchange no data."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return list(range(rank, int(n), world))


def set_devices(devices):
    """Devices host-mode (out-of-core) calls deal their bricks over, round
    robin (brick k on devices[k mod n]); [] = the current device only."""
    devs = [int(d) for d in devices]
    arr = (ctypes.c_int * max(1, len(devs)))(*devs)
    check(lib.hp_set_devices(arr, len(devs)))


def get_devices() -> list:
    n = ctypes.c_int(0)
    check(lib.hp_get_devices(None, 0, ctypes.byref(n)))
    arr = (ctypes.c_int * max(1, n.value))()
    check(lib.hp_get_devices(arr, n.value, ctypes.byref(n)))
    return list(arr[:n.value])


def set_brick_shard(rank: int, world: int):
    """Host-mode calls of this process run only bricks i with i mod world ==
    rank (and write only their cores); (0, 1) runs every brick."""
    check(lib.hp_set_brick_shard(int(rank), int(world)))


def set_memory_budget(nbytes: int):
    check(lib.hp_set_memory_budget(int(nbytes)))


def get_memory_budget() -> int:
    v = ctypes.c_size_t(0)
    check(lib.hp_get_memory_budget(ctypes.byref(v)))
    return v.value


def stream_status(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    check(lib.hp_stream_status(ctypes.c_void_p(s.cuda_stream)))


def selftest_wait_timeout(stream=None):
    """Enqueue a kernel whose bounded device-side wait runs out (diagnostic of
    the failure path); the next stream_status() raises HP_ERR_TIMEOUT."""
    s = stream if stream is not None else torch.cuda.current_stream()
    check(lib.hp_selftest_wait_timeout(ctypes.c_void_p(s.cuda_stream)))


def probe_fp32_fma(repeats: int = 5, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (FLOP/s)."""
    s = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double(0.0)
    check(lib.hp_probe_fp32_fma(ctypes.c_void_p(s.cuda_stream), int(repeats), ctypes.byref(v)))
    return v.value


def stats() -> dict:
    s = hp_stats()
    check(lib.hp_get_stats(ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in hp_stats._fields_}


def release_cache():
    check(lib.hp_release_cache())


def version() -> str:
    return lib.hp_version().decode()
