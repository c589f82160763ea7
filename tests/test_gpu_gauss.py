"""GPU parity: separable Gaussian / derivative filters through the C ABI
against the FP64 oracle (max |err| <= 1e-4 x range), and chunked
(out-of-core, halo-padded bricks) == unchunked bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SHAPES = [(7, 9, 11), (33, 45, 70), (40, 64, 64), (5, 3, 2), (70, 33, 96)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
def test_gaussian_parity_dtypes(shape, dtype):
    f = rand_volume(dtype, shape, 1)
    for sigma, order in [(1.0, (0, 0, 0)), (2.0, (0, 1, 2)), (0.7, (1, 0, 0))]:
        got = to_np(hp.gaussian3d(to_dev(f), sigma, order))
        ref = oracle.gaussian3d(f, sigma, order)
        assert_filter_close(got, ref, f"{dtype.__name__} {shape} s={sigma} o={order}")


@pytest.mark.parametrize("sigma", [0.7, 1.0, 1.5, 2.0, 3.0, 4.0, 5.0, 7.0])
def test_gaussian_parity_radii(sigma):
    """r = 2..12 on the tiled kernel, r = 15 and 21 on the generic path."""
    f = synth.porous((40, 48, 64), 3)[0]
    for order in [(0, 0, 0), (2, 1, 0)]:
        got = to_np(hp.gaussian3d(to_dev(f), sigma, order))
        ref = oracle.gaussian3d(f, sigma, order)
        assert_filter_close(got, ref, f"s={sigma} o={order}")


def test_gaussian_f16_output():
    f = synth.porous_f16((24, 40, 64), 4)
    got = to_np(hp.gaussian3d(to_dev(f), 1.0, (0, 0, 1), out_dtype=hp.HP_F16))
    assert got.dtype == np.float16
    assert_filter_close(got, oracle.gaussian3d(f, 1.0, (0, 0, 1)), "f16 out")


def test_gaussian_spheres_config_128():
    f = synth.spheres(128, 40, synth.SEED_BASE + 0)
    got = to_np(hp.gaussian3d(to_dev(f), 2.0))
    assert_filter_close(got, oracle.gaussian3d(f, 2.0), "128^3 sigma 2")


@pytest.mark.parametrize("sigma,order", [(1.0, (0, 0, 0)), (3.0, (0, 0, 0)), (2.0, (1, 1, 0))])
def test_chunked_equals_unchunked_bitwise(sigma, order):
    f = synth.porous((96, 80, 72), 5)[0]
    whole = to_np(hp.gaussian3d(to_dev(f), sigma, order))
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(3 * (80 * 72 * 40) * 6)      # ~a dozen z slabs
        host_out = np.empty(f.shape, np.float32)
        hp.gaussian3d(f, sigma, order, out=host_out)
        st = hp.stats()
        assert st["bricks"] >= 3
        assert st["peak_device_bytes"] <= st["budget_bytes"]
        assert st["live_device_bytes"] == 0
    finally:
        hp.set_memory_budget(old)
    assert np.array_equal(host_out.view(np.uint32), whole.view(np.uint32))


def test_chunked_xy_split_equals_unchunked_bitwise():
    f = rand_volume(np.float32, (6, 200, 160), 7)
    whole = to_np(hp.gaussian3d(to_dev(f), 2.0))
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(3 * 500_000)        # one plane + halos (768 KB) does not fit
        pinned = torch.from_numpy(f).pin_memory()
        out = torch.empty(f.shape, dtype=torch.float32).pin_memory()
        hp.gaussian3d(pinned, 2.0, out=out)
        assert hp.stats()["bricks"] > 6
    finally:
        hp.set_memory_budget(old)
    assert np.array_equal(out.numpy().view(np.uint32), whole.view(np.uint32))


def test_full_size_sampled_parity_1024():
    """The workload bench.py times: 1024^3 uint16 porous, sigma 1, 2, 4;
    sampled 8^3 boxes (corners, faces, random) against the oracle."""
    n = 1024
    f, _ = synth.porous(n, synth.SEED_BASE + 1)
    x = to_dev(f)
    boxes = [(0, 0, 0), (n - 8, n - 8, n - 8), (0, n - 8, 500), (512, 0, n - 8), (333, 777, 3)]
    rng = np.random.default_rng(0)
    boxes += [tuple(int(v) for v in rng.integers(0, n - 8, 3)) for _ in range(3)]
    for sigma in (1.0, 2.0, 4.0):
        y = hp.gaussian3d(x, sigma)
        torch.cuda.synchronize()
        r = oracle.radius(sigma)
        refs, gots = [], []
        for lo in boxes:
            ilo = [max(0, c - r) for c in lo]
            ihi = [min(n, c + 8 + r) for c in lo]
            # reflected sources of a face box lie inside [0, 8 + r)
            part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
            refs.append(oracle.gaussian3d(part, sigma, gdims=f.shape, in_lo=ilo, out_lo=lo,
                                          out_shape=(8, 8, 8)))
            gots.append(y[lo[0]:lo[0] + 8, lo[1]:lo[1] + 8, lo[2]:lo[2] + 8].cpu().numpy())
        # the range over the sampled boxes is a lower bound of the full range,
        # so this tolerance is at most the 1e-4 x range bar
        ref = np.stack(refs)
        assert_filter_close(np.stack(gots), ref, f"1024^3 sigma {sigma}")
        del y


def test_full_size_face_planes_and_interior_block_1024():
    """The 1024^3 step's Gaussians on whole face planes (z = 0, y = n - 1,
    x = 0: every face tile path and the reflected z groups) and one interior
    64^3 block (several tiles and z chunks in full), against the oracle
    (its OpenMP build: the same operations in the same order)."""
    n = 1024
    f, _ = synth.porous(n, synth.SEED_BASE + 1)
    x = to_dev(f)
    oracle.use_threads(True)
    try:
        for sigma in (1.0, 2.0, 4.0):
            y = hp.gaussian3d(x, sigma)
            torch.cuda.synchronize()
            r = oracle.radius(sigma)
            boxes = [((0, 0, 0), (1, n, n)), ((0, n - 1, 0), (n, 1, n)), ((0, 0, 0), (n, n, 1)),
                     ((480, 300, 700), (64, 64, 64))]
            for lo, shp in boxes:
                ilo = [max(0, c - r) for c in lo]
                ihi = [min(n, c + s + r) for c, s in zip(lo, shp)]
                part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
                ref = oracle.gaussian3d(part, sigma, gdims=f.shape, in_lo=ilo, out_lo=lo,
                                        out_shape=shp)
                got = y[lo[0]:lo[0] + shp[0], lo[1]:lo[1] + shp[1], lo[2]:lo[2] + shp[2]]
                assert_filter_close(got.cpu().numpy(), ref, f"1024^3 sigma {sigma} box {lo}+{shp}")
            del y
    finally:
        oracle.use_threads(False)
