"""GPU parity of two exact decisions against the oracle, bit for bit:

- erosion, dilation and the morphology subgradient order floating-point
  values by IEEE 754 totalOrder (-0 below +0, +NaN above +inf, -NaN below
  -inf), on float16 and float32 volumes full of signed-zero ties,
  infinities and NaNs;
- the global threshold decides f > t exactly for thresholds that are not
  representable in the input's type (they round up or down), for every
  input dtype.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SE_NAME = {oracle.SE_CUBE: "cube", oracle.SE_BALL: "ball"}

F32_SPECIALS = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000,
                         0x7FC00001, 0xFFC00001, 0x3F800000, 0xBF800000, 0x00000001, 0x80000001],
                        np.uint32)
F16_SPECIALS = np.array([0x0000, 0x8000, 0x7C00, 0xFC00, 0x7E00, 0xFE00, 0x7E01, 0xFE01, 0x3C00,
                         0xBC00, 0x0001, 0x8001], np.uint16)


def _special_volume(dtype, shape, seed, frac):
    """Mostly +-0 (ties of the two zeros everywhere), with a fraction of
    infinities, NaNs of both signs and payloads, and small values."""
    rng = np.random.default_rng(seed)
    sp = F32_SPECIALS if dtype == np.float32 else F16_SPECIALS
    zeros = sp[:2]
    bits = rng.choice(zeros, shape)
    m = rng.random(shape) < frac
    bits[m] = rng.choice(sp, int(m.sum()))
    return bits.view(dtype)


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint16)


@pytest.mark.parametrize("dtype", [np.float16, np.float32])
@pytest.mark.parametrize("shape", [(9, 13, 64), (12, 33, 72), (6, 5, 8)])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_BALL, 2), (oracle.SE_BALL, 3),
                                    (oracle.SE_CUBE, 4), (oracle.SE_CUBE, 8), (oracle.SE_BALL, 7)])
def test_morph_total_order(dtype, shape, se, rad):
    for frac in (0.02, 0.3):
        f = _special_volume(dtype, shape, 3 + rad, frac)
        x = to_dev(f)
        e = to_np(hp.erode3d(x, SE_NAME[se], rad))
        d = to_np(hp.dilate3d(x, SE_NAME[se], rad))
        assert np.array_equal(_bits(e), _bits(oracle.erode3d(f, se, rad))), "erode"
        assert np.array_equal(_bits(d), _bits(oracle.dilate3d(f, se, rad))), "dilate"


@pytest.mark.parametrize("dtype", [np.float16, np.float32])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_CUBE, 2), (oracle.SE_BALL, 2)])
@pytest.mark.parametrize("dilate", [False, True])
def test_subgradient_total_order(dtype, se, rad, dilate):
    """The subgradient routes every output to the source the forward copied
    (totalOrder, ties to the smallest linear index): the summed gradients
    match the oracle's exactly, since each voxel sums its routed weights in
    the same increasing order (weights are small integers, so the sums are
    exact in FP32 as well)."""
    shape = (10, 12, 40)
    f = _special_volume(dtype, shape, 9, 0.1)
    rng = np.random.default_rng(10)
    w = rng.integers(-8, 9, shape).astype(np.float32)
    g = hp.morph3d_backward(to_dev(f), to_dev(w), dilate, SE_NAME[se], rad)
    ref = oracle.morph3d_vjp(f, se, rad, dilate, w.astype(np.float64))
    assert np.array_equal(to_np(g).astype(np.float64), ref)


THRESHOLDS = [0.1, 0.5, 1.0 / 3.0, 7499.7, 7499.9999999, 65535.5, -0.0, 0.0, -1.5, 1e30, -1e30,
              float(np.float32(0.1)), float(np.nextafter(np.float32(0.1), np.float32(0)))]


def _neighbours(dtype, ts, vals):
    for t in ts:
        if dtype in (np.uint8, np.uint16):
            top = np.iinfo(dtype).max
            c = int(np.floor(t)) if abs(t) < 1e9 else (0 if t < 0 else top)
            vals += [v for v in range(c - 2, c + 3) if 0 <= v <= top]
        else:
            c = np.array(t, dtype)
            a = c
            for _ in range(3):
                vals.append(a)
                a = np.nextafter(a, dtype(np.inf))
            a = c
            for _ in range(3):
                a = np.nextafter(a, dtype(-np.inf))
                vals.append(a)


def _neighbour_volume(dtype, ts):
    """Every representable neighbour of each threshold (the values just
    below, at and above it in the input's type), plus random values."""
    vals = []
    with np.errstate(over="ignore"):
        _neighbours(dtype, ts, vals)
    rng = np.random.default_rng(4)
    base = (rng.integers(0, 256 if dtype == np.uint8 else 65536, 4096) if dtype in (np.uint8, np.uint16)
            else rng.standard_normal(4096) * 4000)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan] if dtype in (np.float16, np.float32) else [0]
    v = np.concatenate([np.array(vals, dtype), base.astype(dtype), np.array(special, dtype)])
    v = np.resize(v, 8 * 16 * 64)
    return v.reshape(8, 16, 64)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
def test_threshold_is_exact_for_unrepresentable_t(dtype):
    f = _neighbour_volume(dtype, THRESHOLDS + [65504.5, 65519.0, 65520.0, 1e6, -7e4])
    x = to_dev(f)
    for t in THRESHOLDS + [65504.5, 65519.0, 65520.0, 1e6, -7e4, float("inf"), float("-inf")]:
        got = to_np(hp.threshold3d(x, t))
        assert np.array_equal(got, oracle.threshold(f, t)), (dtype, t)


def test_threshold_rejects_nan():
    x = torch.zeros((2, 2, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(hp.HPError):
        hp.threshold3d(x, float("nan"))
