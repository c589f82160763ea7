"""Seeded synthetic inputs for the chunked 3D filtering workloads.

This package draws input volumes, weight fields and brick partitions. It
holds none of the method's arithmetic; the CPU oracle and the CUDA library
both consume what it returns. The C source (``synth.c``) is compiled into
``libsynth.so`` next to it on first use (``build()``).

Workload recipes (seed = 2511118900 + k for workload k):
  - ``spheres(n, count, seed)``: float32 balls of 1.0 on 0.2 plus N(0, 0.05^2).
  - ``porous(n, seed)``: uint16 porous tomogram, 35% pores, 12000/3000
    Poisson-like intensities, 1% linear gradient along z.
  - ``porous_f16(n, seed)``: the same volume scaled by 1/65535, stored as float16.
  - ``normal_field(shape, seed)``: float32 N(0, 1) weights.
  - ``kd_bricks(...)``: seeded k-d partition of a volume into disjoint boxes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_BASE = 2511118900


def build(force: bool = False) -> str:
    """Compile libsynth.so (gcc, OpenMP) if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.synth_spheres_f32.argtypes = [vp, i64, i64, i64, i64, u64]
        lib.synth_spheres_f32.restype = ctypes.c_int
        lib.synth_porous_u16.argtypes = [vp, i64, i64, i64, u64, ctypes.POINTER(ctypes.c_double)]
        lib.synth_porous_u16.restype = ctypes.c_int
        lib.synth_porous_count.argtypes = [i64, i64, i64, ctypes.c_double]
        lib.synth_porous_count.restype = i64
        lib.synth_normal_f32.argtypes = [vp, i64, u64]
        lib.synth_normal_f64.argtypes = [vp, i64, u64]
        lib.synth_kd_bricks.argtypes = [vp, ctypes.c_int, i64, i64, i64, i64, i64, u64]
        lib.synth_kd_bricks.restype = ctypes.c_int
        lib.synth_pick.argtypes = [vp, i64, i64, u64]
        lib.synth_uniform.argtypes = [u64, ctypes.c_int, u64]
        lib.synth_uniform.restype = ctypes.c_double
        lib.synth_normal.argtypes = [u64, ctypes.c_int, u64]
        lib.synth_normal.restype = ctypes.c_double
        lib.synth_draw_u64.argtypes = [u64, ctypes.c_int, u64]
        lib.synth_draw_u64.restype = u64
        _lib = lib
    return _lib


def _shape3(n):
    if isinstance(n, int):
        return (n, n, n)
    nz, ny, nx = n
    return (int(nz), int(ny), int(nx))


def spheres(n, count: int, seed: int, out: np.ndarray | None = None) -> np.ndarray:
    """float32 (nz, ny, nx) volume of `count` value-1.0 balls on 0.2, plus noise."""
    nz, ny, nx = _shape3(n)
    if out is None:
        out = np.empty((nz, ny, nx), np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.shape == (nz, ny, nx)
    if _load().synth_spheres_f32(out.ctypes.data, nx, ny, nz, count, seed) != 0:
        raise MemoryError("synth_spheres_f32")
    return out


def porous(n, seed: int, out: np.ndarray | None = None) -> tuple[np.ndarray, float]:
    """uint16 (nz, ny, nx) porous tomogram; returns (volume, drawn porosity)."""
    nz, ny, nx = _shape3(n)
    if out is None:
        out = np.empty((nz, ny, nx), np.uint16)
    assert out.dtype == np.uint16 and out.flags.c_contiguous and out.shape == (nz, ny, nx)
    por = ctypes.c_double(0.0)
    if _load().synth_porous_u16(out.ctypes.data, nx, ny, nz, seed, ctypes.byref(por)) != 0:
        raise MemoryError("synth_porous_u16")
    return out, por.value


def porous_count(n, porosity: float = 0.35) -> int:
    nz, ny, nx = _shape3(n)
    return int(_load().synth_porous_count(nx, ny, nz, porosity))


def porous_f16(n, seed: int) -> np.ndarray:
    """The porous volume scaled by 1/65535 and rounded to float16."""
    v, _ = porous(n, seed)
    return (v.astype(np.float32) * np.float32(1.0 / 65535.0)).astype(np.float16)


def normal_field(shape, seed: int, dtype=np.float32) -> np.ndarray:
    out = np.empty(tuple(shape), dtype)
    n = out.size
    if dtype == np.float32:
        _load().synth_normal_f32(out.ctypes.data, n, seed)
    elif dtype == np.float64:
        _load().synth_normal_f64(out.ctypes.data, n, seed)
    else:
        raise TypeError(dtype)
    return out


def kd_bricks(n, nbricks: int, seed: int, minside: int = 64, quantum: int = 16) -> np.ndarray:
    """(nbricks, 6) int64 boxes [z0, y0, x0, z1, y1, x1] partitioning the volume."""
    nz, ny, nx = _shape3(n)
    boxes = np.zeros((nbricks, 6), np.int64)
    got = _load().synth_kd_bricks(boxes.ctypes.data, nbricks, nx, ny, nz, minside, quantum, seed)
    if got < 0:
        raise ValueError("bad kd_bricks arguments")
    return boxes[:got].copy()


def pick(m: int, n: int, seed: int) -> np.ndarray:
    """m uniform linear indices in [0, n)."""
    out = np.empty(m, np.int64)
    _load().synth_pick(out.ctypes.data, m, n, seed)
    return out


def uniform(seed: int, stream: int, i: int) -> float:
    return _load().synth_uniform(seed, stream, i)


def draw_u64(seed: int, stream: int, i: int) -> int:
    return _load().synth_draw_u64(seed, stream, i)
