"""CPU oracle for chunked 3D Gaussian / derivative / morphology filtering.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library. It wraps the
plain single-threaded FP64 C in ``oracle.c`` (compiled to ``liboracle.so``
next to it, with ``-ffp-contract=off`` so every product and sum rounds in
FP64 as written) and shares no code with the CUDA path.

Each function follows the paper's filter list (Sec. III-C: Gaussian,
"Hessian" feature extraction, erosion, dilation, threshold) and its chunked
execution model (Sec. III-D: overlapping, context-preserving Z chunks). The
paper prints no formulas; the conventions written in ``oracle.c`` are the
readings this project fixes. Arrays are numpy, C order, shape (nz, ny, nx).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against scipy.ndimage (an independent library), closed forms, invariants or
brute force on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_MT = os.path.join(_HERE, "liboracle_mt.so")
_lib = None
_libs = {}

U8, U16, F16, F32, F64 = 0, 1, 2, 3, 4
SE_CUBE, SE_BALL = 0, 1
G, GM, LOG = 0, 1, 2
_DT = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float16): F16,
       np.dtype(np.float32): F32, np.dtype(np.float64): F64}
_ERR = {-1: "bad argument", -2: "out of memory", -3: "input box misses a needed voxel (halo too small)"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False, threads: bool = False) -> str:
    """Compile liboracle.so (single-threaded) or, with threads=True,
    liboracle_mt.so (the same source with -fopenmp) if missing or stale."""
    out = _LIB_MT if threads else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", *(["-fopenmp"] if threads else []), "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, out)
    return out


def use_threads(on: bool):
    """Route the functions below to the OpenMP build (on) or the
    single-threaded build (off, the default); results are identical."""
    global _lib
    _lib = _open(bool(on))


def _load():
    global _lib
    if _lib is None:
        _lib = _open(False)
    return _lib


def _open(threads: bool):
    if threads not in _libs:
        lib = ctypes.CDLL(build(threads=threads))
        vp, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        p3 = ctypes.POINTER(ctypes.c_int64)
        lib.orc_reflect.argtypes = [i64, i64]
        lib.orc_reflect.restype = i64
        lib.orc_radius.argtypes = [d, d]
        lib.orc_radius.restype = i
        lib.orc_kernel1d.argtypes = [d, i, i, vp]
        lib.orc_gaussian3d.argtypes = [vp, i, p3, p3, p3, p3, p3, d, d, vp, vp]
        lib.orc_filterbank3d.argtypes = [vp, i, p3, p3, p3, p3, p3, vp, vp, i, d, vp]
        lib.orc_morph3d.argtypes = [vp, i, p3, p3, p3, p3, p3, i, i, i, vp]
        lib.orc_threshold.argtypes = [vp, i, i64, d, vp]
        lib.orc_gaussian3d_adjoint.argtypes = [vp, p3, d, d, vp, vp]
        lib.orc_filterbank3d_vjp.argtypes = [vp, i, p3, vp, vp, i, d, vp, vp]
        lib.orc_morph3d_vjp.argtypes = [vp, i, p3, i, i, i, vp, vp, vp]
        lib.orc_box_sums.argtypes = [vp, i, p3, i, vp, vp]
        lib.orc_threshold_box.argtypes = [vp, i, p3, i, i, d, d, vp, vp]
        _libs[threads] = lib
    return _libs[threads]


def _check(rc: int):
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))


def _v3(t):
    return (ctypes.c_int64 * 3)(*[int(v) for v in t])


def _in(a: np.ndarray):
    a = np.ascontiguousarray(a)
    if a.dtype not in _DT or a.ndim != 3:
        raise TypeError(f"oracle input must be a 3D array of u8/u16/f16/f32/f64, got {a.dtype}")
    return a, _DT[a.dtype]


def reflect(i: int, n: int) -> int:
    return int(_load().orc_reflect(i, n))


def radius(sigma: float, truncate: float = 3.0) -> int:
    return int(_load().orc_radius(sigma, truncate))


def kernel1d(sigma: float, order: int = 0, truncate: float = 3.0) -> np.ndarray:
    """FP64 taps g_order(k), k = -r..r (index k + r)."""
    r = radius(sigma, truncate)
    w = np.empty(2 * r + 1, np.float64)
    _check(_load().orc_kernel1d(sigma, r, order, w.ctypes.data))
    return w


def _boxes(vol_shape, gdims, in_lo, out_lo, out_shape):
    gdims = tuple(vol_shape) if gdims is None else tuple(gdims)
    in_lo = (0, 0, 0) if in_lo is None else tuple(in_lo)
    out_lo = (0, 0, 0) if out_lo is None else tuple(out_lo)
    out_shape = tuple(gdims) if out_shape is None else tuple(out_shape)
    return gdims, in_lo, out_lo, out_shape


def gaussian3d(f: np.ndarray, sigma: float, order=(0, 0, 0), truncate: float = 3.0, *,
               gdims=None, in_lo=None, out_lo=None, out_shape=None) -> np.ndarray:
    """FP64 Gaussian (or derivative of orders (oz, oy, ox)) with reflect boundary.

    By default ``f`` is the whole volume and the whole output is returned.
    For chunked use, ``f`` is the input box at ``in_lo`` of a global volume
    of shape ``gdims``, and the output covers ``out_shape`` at ``out_lo``.
    """
    f, dt = _in(f)
    gdims, in_lo, out_lo, out_shape = _boxes(f.shape, gdims, in_lo, out_lo, out_shape)
    out = np.empty(out_shape, np.float64)
    ordv = (ctypes.c_int * 3)(*order)
    _check(_load().orc_gaussian3d(f.ctypes.data, dt, _v3(in_lo), _v3(f.shape), _v3(gdims),
                                  _v3(out_lo), _v3(out_shape), float(sigma), float(truncate),
                                  ordv, out.ctypes.data))
    return out


def filterbank3d(f: np.ndarray, filters, truncate: float = 3.0, *, gdims=None, in_lo=None,
                 out_lo=None, out_shape=None) -> list[np.ndarray]:
    """FP64 outputs of filters [(kind, sigma), ...], kind in {G, GM, LOG}."""
    f, dt = _in(f)
    gdims, in_lo, out_lo, out_shape = _boxes(f.shape, gdims, in_lo, out_lo, out_shape)
    n = len(filters)
    outs = [np.empty(out_shape, np.float64) for _ in range(n)]
    kinds = (ctypes.c_int * n)(*[int(k) for k, _ in filters])
    sig = (ctypes.c_double * n)(*[float(s) for _, s in filters])
    ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    _check(_load().orc_filterbank3d(f.ctypes.data, dt, _v3(in_lo), _v3(f.shape), _v3(gdims),
                                    _v3(out_lo), _v3(out_shape), kinds, sig, n, float(truncate),
                                    ptrs))
    return outs


def morph3d(f: np.ndarray, se: int, rad: int, dilate: bool, *, gdims=None, in_lo=None,
            out_lo=None, out_shape=None) -> np.ndarray:
    """Exact grayscale erosion (dilate=False) or dilation, output in f's dtype."""
    f, dt = _in(f)
    gdims, in_lo, out_lo, out_shape = _boxes(f.shape, gdims, in_lo, out_lo, out_shape)
    out = np.empty(out_shape, f.dtype)
    _check(_load().orc_morph3d(f.ctypes.data, dt, _v3(in_lo), _v3(f.shape), _v3(gdims),
                               _v3(out_lo), _v3(out_shape), int(se), int(rad), int(bool(dilate)),
                               out.ctypes.data))
    return out


def erode3d(f, se, rad, **kw):
    return morph3d(f, se, rad, False, **kw)


def dilate3d(f, se, rad, **kw):
    return morph3d(f, se, rad, True, **kw)


def open3d(f, se, rad):
    """Opening (Sec. III-C morphology): dilation of the erosion, each with
    reflect boundaries over the whole volume."""
    return dilate3d(erode3d(f, se, rad), se, rad)


def close3d(f, se, rad):
    """Closing: erosion of the dilation."""
    return erode3d(dilate3d(f, se, rad), se, rad)


def tophat3d(f, se, rad):
    """White top-hat: f minus its opening, rounded once (to nearest, ties to
    even) to f's dtype. Integers: exact, since f >= its opening. float16:
    the difference of two float16 values is exact in FP64 (both are
    multiples of 2^-24 below 2^16 in magnitude, so it needs at most 41
    significant bits), then one rounding to float16. float32: the FP32
    subtraction itself (correctly rounded). float64: the FP64 subtraction."""
    o = open3d(f, se, rad)
    if f.dtype == np.float32:
        return f - o
    return (f.astype(np.float64) - o.astype(np.float64)).astype(f.dtype)


def unsharp3d(f, sigma, amount):
    """Unsharp mask f + amount * (f - G_sigma f) in FP64 (the Gaussian as
    gaussian3d: truncate 3, reflect)."""
    x = f.astype(np.float64)
    return x + amount * (x - gaussian3d(f, sigma))


def threshold_local(f: np.ndarray, sigma: float, offset: float = 0.0):
    """Gaussian local threshold (Sec. III-C threshold algorithms): the
    decision f > T with T = G_sigma f - offset in FP64; returns (u8 decision,
    T) so that a test can tell decisions that FP32 rounding may flip (f
    within the Gaussian's error bar of T) from those it may not."""
    t = gaussian3d(f, sigma) - offset
    return (f.astype(np.float64) > t).astype(np.uint8), t


LOCAL_MEAN, LOCAL_NIBLACK, LOCAL_SAUVOLA = 0, 1, 2


def box_sums(f: np.ndarray, w: int):
    """FP64 window sums of f and f^2 over the (2w+1)^3 cube, reflect
    boundary, accumulated x then y then z in increasing source coordinate."""
    f, dt = _in(f)
    s1 = np.empty(f.shape, np.float64)
    s2 = np.empty(f.shape, np.float64)
    _check(_load().orc_box_sums(f.ctypes.data, dt, _v3(f.shape), int(w), s1.ctypes.data,
                                s2.ctypes.data))
    return s1, s2


def threshold_box(f: np.ndarray, method: int, w: int, k: float = 0.0, c: float = 0.0,
                  return_threshold: bool = False):
    """Local threshold over a (2w+1)^3 box window (Sec. III-C threshold
    algorithms: mean, Niblack, Sauvola), decided in FP64: u8 = f > T with
    T = m - c (mean), m + k s (Niblack) or m (1 + k (s / c - 1)) (Sauvola,
    c = R), m and s the window mean and standard deviation."""
    f, dt = _in(f)
    out = np.empty(f.shape, np.uint8)
    thr = np.empty(f.shape, np.float64) if return_threshold else None
    _check(_load().orc_threshold_box(f.ctypes.data, dt, _v3(f.shape), int(method), int(w),
                                     float(k), float(c), out.ctypes.data,
                                     thr.ctypes.data if return_threshold else None))
    return (out, thr) if return_threshold else out


HESSIAN_ORDERS = ((2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1))


def hessian3d(f: np.ndarray, sigma: float):
    """The six distinct entries of the Hessian of the Gaussian-smoothed
    volume (Sec. III-C "Hessian" texture features), FP64, in the order
    Dzz, Dyy, Dxx, Dzy, Dzx, Dyx: each the Gaussian derivative filter of
    orders (oz, oy, ox) summing to 2."""
    return [gaussian3d(f, sigma, o) for o in HESSIAN_ORDERS]


def hessian_eigenvalues(f: np.ndarray, sigma: float):
    """Eigenvalues of the symmetric 3x3 Hessian per voxel, ascending
    (l1 <= l2 <= l3), in FP64: the matrix assembled from hessian3d and
    numpy.linalg.eigvalsh (LAPACK's symmetric eigensolver) as the step."""
    zz, yy, xx, zy, zx, yx = hessian3d(f, sigma)
    h = np.stack([np.stack([zz, zy, zx], -1), np.stack([zy, yy, yx], -1),
                  np.stack([zx, yx, xx], -1)], -2)
    ev = np.linalg.eigvalsh(h)
    return [np.ascontiguousarray(ev[..., i]) for i in range(3)]


def threshold(f: np.ndarray, t: float = 0.5) -> np.ndarray:
    f = np.ascontiguousarray(f)
    out = np.empty(f.shape, np.uint8)
    _check(_load().orc_threshold(f.ctypes.data, _DT[f.dtype], f.size, float(t), out.ctypes.data))
    return out


def gaussian3d_adjoint(w: np.ndarray, sigma: float, order=(0, 0, 0),
                       truncate: float = 3.0) -> np.ndarray:
    """A^T w for A = gaussian3d(., sigma, order) on the whole volume."""
    w = np.ascontiguousarray(w, np.float64)
    g = np.empty_like(w)
    ordv = (ctypes.c_int * 3)(*order)
    _check(_load().orc_gaussian3d_adjoint(w.ctypes.data, _v3(w.shape), float(sigma),
                                          float(truncate), ordv, g.ctypes.data))
    return g


def filterbank3d_vjp(f: np.ndarray, filters, ws, truncate: float = 3.0) -> np.ndarray:
    """sum_i J_i^T w_i for the filter bank at input f (whole volume)."""
    f, dt = _in(f)
    n = len(filters)
    ws = [np.ascontiguousarray(w, np.float64) for w in ws]
    g = np.empty(f.shape, np.float64)
    kinds = (ctypes.c_int * n)(*[int(k) for k, _ in filters])
    sig = (ctypes.c_double * n)(*[float(s) for _, s in filters])
    ptrs = (ctypes.c_void_p * n)(*[w.ctypes.data for w in ws])
    _check(_load().orc_filterbank3d_vjp(f.ctypes.data, dt, _v3(f.shape), kinds, sig, n,
                                        float(truncate), ptrs, g.ctypes.data))
    return g


def morph3d_vjp(f: np.ndarray, se: int, rad: int, dilate: bool, w: np.ndarray,
                return_arg: bool = False):
    """Subgradient of sum(w * morph(f)) w.r.t. f, ties to the smallest source index."""
    f, dt = _in(f)
    w = np.ascontiguousarray(w, np.float64)
    g = np.empty(f.shape, np.float64)
    arg = np.empty(f.shape, np.int64) if return_arg else None
    _check(_load().orc_morph3d_vjp(f.ctypes.data, dt, _v3(f.shape), int(se), int(rad),
                                   int(bool(dilate)), w.ctypes.data, g.ctypes.data,
                                   arg.ctypes.data if return_arg else None))
    return (g, arg) if return_arg else g
