"""GPU parity of the Hessian features and the box-window local thresholds
(Sec. III-C) through the C ABI, device and host (out-of-core) volumes.

- Hessian components: the Gaussian derivative kernels, within the FP32
  filter bar (1e-4 x the range of each FP64 component).
- Hessian eigenvalues: by Weyl's inequality an eigenvalue moves by at most
  the spectral norm of the perturbation, which is at most the sum of the
  component errors; the bar is therefore 1e-4 x (sum of the component
  ranges), plus the FP32 closed-form solve (a few ulp of the largest
  entry).
- Mean / Niblack / Sauvola decisions: bit-exact for every input dtype (the
  window sums and the FP64 decision run the same operations in the same
  order as the oracle).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")


@pytest.mark.parametrize("shape", [(20, 33, 40), (9, 12, 70)])
@pytest.mark.parametrize("sigma", [1.0, 2.0, 5.0])
def test_hessian_components(shape, sigma):
    f = synth.porous(shape, 51)[0]
    got = [to_np(t) for t in hp.hessian3d(to_dev(f), sigma)]
    for g, r in zip(got, oracle.hessian3d(f, sigma)):
        assert_filter_close(g, r, f"Hessian sigma {sigma}")


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.float16])
@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_hessian_eigenvalues(dtype, sigma):
    f = synth.porous((24, 36, 48), 52)[0]
    if dtype != np.uint16:
        f = (f.astype(np.float64) / 65535.0).astype(dtype)
    got = [to_np(t) for t in hp.hessian3d(to_dev(f), sigma, eigenvalues=True)]
    comps = oracle.hessian3d(f, sigma)
    ref = oracle.hessian_eigenvalues(f, sigma)
    bar = 1e-4 * sum(float(c.max() - c.min()) for c in comps)
    bar += 8 * np.finfo(np.float32).eps * max(float(np.abs(c).max()) for c in comps)
    for i, (g, r) in enumerate(zip(got, ref)):
        err = np.abs(g.astype(np.float64) - r).max()
        assert err <= bar, (i, err, bar)
    assert (got[0] <= got[1]).all() and (got[1] <= got[2]).all()


def test_hessian_out_of_core_equals_device():
    f = synth.porous((48, 40, 56), 53)[0]
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(12_000_000)
        host = hp.hessian3d(f, 2.0, eigenvalues=True)
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4 and st["peak_device_bytes"] <= 12_000_000 and st["live_device_bytes"] == 0
    dev = [to_np(t) for t in hp.hessian3d(to_dev(f), 2.0, eigenvalues=True)]
    for a, b in zip(host, dev):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


METHODS = [("mean", 0.0, 150.0), ("niblack", 0.2, 0.0), ("niblack", -0.5, 0.0), ("sauvola", 0.3, 32768.0),
           ("sauvola", 0.5, 0.25)]
MCODE = {"mean": oracle.LOCAL_MEAN, "niblack": oracle.LOCAL_NIBLACK, "sauvola": oracle.LOCAL_SAUVOLA}


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("method,k,c", METHODS)
@pytest.mark.parametrize("w", [1, 3])
def test_box_threshold_bit_exact(dtype, method, k, c, w):
    f = rand_volume(dtype, (14, 23, 37), 60 + w)
    if dtype == np.float16:
        f = (np.abs(f.astype(np.float32)) * 0.1).astype(np.float16)
    got = to_np(hp.threshold_box3d(to_dev(f), method, w, k, c))
    ref = oracle.threshold_box(f, MCODE[method], w, k, c)
    assert np.array_equal(got, ref)


def test_box_threshold_porous_and_out_of_core():
    f = synth.porous((40, 64, 72), 61)[0]
    ref = oracle.threshold_box(f, oracle.LOCAL_SAUVOLA, 4, 0.2, 32768.0)
    assert np.array_equal(to_np(hp.threshold_box3d(to_dev(f), "sauvola", 4, 0.2, 32768.0)), ref)
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(8_000_000)
        host = hp.threshold_box3d(f, "sauvola", 4, 0.2, 32768.0)
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4 and st["peak_device_bytes"] <= 8_000_000
    assert np.array_equal(host, ref)


def test_box_threshold_radius_beyond_extent_and_errors():
    f = rand_volume(np.uint16, (3, 2, 5), 7)
    got = to_np(hp.threshold_box3d(to_dev(f), "niblack", 4, 0.1))
    assert np.array_equal(got, oracle.threshold_box(f, oracle.LOCAL_NIBLACK, 4, 0.1, 0.0))
    x = to_dev(f)
    with pytest.raises(hp.HPError, match="HP_ERR_INVALID_ARG"):
        hp.threshold_box3d(x, "sauvola", 2, 0.2, 0.0)
    with pytest.raises(hp.HPError, match="HP_ERR_INVALID_ARG"):
        hp.threshold_box3d(x, "mean", 16)


def test_box_threshold_radius_zero_and_hessian_small_sigma_f16():
    f = rand_volume(np.uint16, (6, 9, 20), 80)
    x = to_dev(f)
    # a 1-voxel window: m = f, s = 0
    assert not to_np(hp.threshold_box3d(x, "niblack", 0, 0.7)).any()          # f > f is false
    assert to_np(hp.threshold_box3d(x, "mean", 0, 0.0, 1.0)).all()             # f > f - 1
    g = rand_volume(np.float32, (10, 12, 16), 81)
    for sigma in (0.4, 0.7):
        got = [to_np(t) for t in hp.hessian3d(to_dev(g), sigma, out_dtype=hp.HP_F16)]
        for a, r in zip(got, oracle.hessian3d(g, sigma)):
            assert_filter_close(a, r, f"Hessian f16 sigma {sigma}")


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_box_threshold_near_ties_and_integer_extremes(dtype):
    """Integer inputs decide in FP32 where f is clear of the threshold and in
    FP64 (the oracle's sequence) otherwise. Piecewise-constant 4^3 blocks with
    sparse +-1 perturbations put many voxels at or next to the threshold
    (windows of zero or tiny variance, f equal to the mean); an all-maximum
    volume at radius 15 takes the window sums to their largest values
    (S1 = 29791 x 65535 < 2^31; the variance numerator N S2 - S1^2 in int64)."""
    rng = np.random.default_rng(90)
    top = np.iinfo(dtype).max
    cases = [("mean", 0.0, 0.0), ("mean", 0.0, 1.0), ("niblack", 0.0, 0.0), ("niblack", 0.5, 0.0),
             ("niblack", -1.0, 0.0), ("sauvola", 0.0, 128.0), ("sauvola", 0.25, float(top) / 2)]
    # 33 columns: element loads along x; 64 columns (whole 16-byte words per
    # row): 16-byte loads for uint16
    for shape in [(15, 22, 33), (12, 20, 64)]:
        blocks = rng.integers(1, top - 1, size=(4, 6, 16))
        f = np.kron(blocks, np.ones((4, 4, 4), np.int64))[:shape[0], :shape[1], :shape[2]]
        bump = rng.random(f.shape)
        f = (f + (bump < 0.05) - (bump > 0.95)).astype(dtype)
        x = to_dev(f)
        for w in (1, 2, 5):
            for method, k, c in cases:
                got = to_np(hp.threshold_box3d(x, method, w, k, c))
                ref = oracle.threshold_box(f, MCODE[method], w, k, c)
                assert np.array_equal(got, ref), (shape, w, method, k, c)
    g = np.full((5, 7, 9), top, dtype)
    g[2, 3, 4] = top - 1
    xg = to_dev(g)
    for method, k, c in [("mean", 0.0, 0.0), ("niblack", 0.3, 0.0), ("sauvola", 0.3, float(top))]:
        got = to_np(hp.threshold_box3d(xg, method, 15, k, c))
        assert np.array_equal(got, oracle.threshold_box(g, MCODE[method], 15, k, c)), method
