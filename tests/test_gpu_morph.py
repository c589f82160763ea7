"""GPU parity: grayscale erosion / dilation and threshold through the C ABI,
bit-exact against the oracle, chunked == unchunked."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SHAPES = [(7, 9, 11), (33, 45, 70), (40, 64, 64), (5, 3, 2)]
SE_NAME = {oracle.SE_CUBE: "cube", oracle.SE_BALL: "ball"}


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_CUBE, 2), (oracle.SE_BALL, 1),
                                    (oracle.SE_BALL, 3)])
def test_morph_parity(shape, dtype, se, rad):
    f = rand_volume(dtype, shape, 2)
    x = to_dev(f)
    e = to_np(hp.erode3d(x, SE_NAME[se], rad))
    d = to_np(hp.dilate3d(x, SE_NAME[se], rad))
    assert np.array_equal(e.view(np.uint8), oracle.erode3d(f, se, rad).view(np.uint8))
    assert np.array_equal(d.view(np.uint8), oracle.dilate3d(f, se, rad).view(np.uint8))


@pytest.mark.parametrize("se,rad", [(oracle.SE_BALL, 2), (oracle.SE_BALL, 4), (oracle.SE_BALL, 5),
                                    (oracle.SE_BALL, 6), (oracle.SE_CUBE, 3), (oracle.SE_CUBE, 6),
                                    (oracle.SE_BALL, 7), (oracle.SE_CUBE, 0), (oracle.SE_BALL, 0)])
def test_morph_radii(se, rad):
    f = synth.porous((30, 50, 64), 6)[0]
    x = to_dev(f)
    assert np.array_equal(to_np(hp.erode3d(x, SE_NAME[se], rad)), oracle.erode3d(f, se, rad))
    assert np.array_equal(to_np(hp.dilate3d(x, SE_NAME[se], rad)), oracle.dilate3d(f, se, rad))


def test_threshold_exact():
    f = synth.spheres(48, 6, 3)
    f.ravel()[:5] = [0.5, np.nextafter(np.float32(0.5), np.float32(1)), 0.49, 0, 1]
    assert np.array_equal(to_np(hp.threshold3d(to_dev(f), 0.5)), oracle.threshold(f, 0.5))
    g = synth.porous((16, 20, 24), 3)[0]
    assert np.array_equal(to_np(hp.threshold3d(to_dev(g), 7500)), oracle.threshold(g, 7500))


def test_spheres_pipeline_128():
    """128^3 spheres: Gaussian sigma 2 -> threshold 0.5 -> erosion and dilation
    with the 3x3x3 cube. Each stage is compared on identical inputs; the
    threshold of the GPU Gaussian agrees with the oracle's except where the
    oracle value lies within the filter tolerance of 0.5."""
    f = synth.spheres(128, 40, synth.SEED_BASE + 0)
    g = hp.gaussian3d(to_dev(f), 2.0)
    b = hp.threshold3d(g, 0.5)
    e = to_np(hp.erode3d(b, "cube", 1))
    d = to_np(hp.dilate3d(b, "cube", 1))
    gh, bh = to_np(g), to_np(b)
    assert np.array_equal(bh, oracle.threshold(gh, 0.5))
    assert np.array_equal(e, oracle.erode3d(bh, oracle.SE_CUBE, 1))
    assert np.array_equal(d, oracle.dilate3d(bh, oracle.SE_CUBE, 1))
    gref = oracle.gaussian3d(f, 2.0)
    tol = 1e-4 * (gref.max() - gref.min())
    clear = np.abs(gref - 0.5) > tol
    assert np.array_equal(bh[clear], (gref[clear] > 0.5).astype(np.uint8))
    assert clear.mean() > 0.999


@pytest.mark.parametrize("se,rad,dil", [(oracle.SE_BALL, 3, False), (oracle.SE_BALL, 5, True),
                                        (oracle.SE_CUBE, 2, True)])
def test_morph_chunked_equals_unchunked(se, rad, dil):
    f = synth.porous((90, 64, 80), 8)[0]
    fn = hp.dilate3d if dil else hp.erode3d
    whole = to_np(fn(to_dev(f), SE_NAME[se], rad))
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(3 * 64 * 80 * 30 * 4)
        out = np.empty_like(f)
        fn(f, SE_NAME[se], rad, out=out)
        assert hp.stats()["bricks"] >= 3
    finally:
        hp.set_memory_budget(old)
    assert np.array_equal(out, whole)


def test_full_size_sampled_ball3_1024():
    n = 1024
    f, _ = synth.porous(n, synth.SEED_BASE + 1)
    x = to_dev(f)
    rad = 3
    rng = np.random.default_rng(1)
    boxes = [(0, 0, 0), (n - 8, n - 8, n - 8), (0, 1000, 17)]
    boxes += [tuple(int(v) for v in rng.integers(0, n - 8, 3)) for _ in range(4)]
    for fn, dil in ((hp.erode3d, False), (hp.dilate3d, True)):
        y = fn(x, "ball", rad)
        torch.cuda.synchronize()
        for lo in boxes:
            ilo = [max(0, c - rad) for c in lo]
            ihi = [min(n, c + 8 + rad) for c in lo]
            part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
            ref = oracle.morph3d(part, oracle.SE_BALL, rad, dil, gdims=f.shape, in_lo=ilo,
                                 out_lo=lo, out_shape=(8, 8, 8))
            got = y[lo[0]:lo[0] + 8, lo[1]:lo[1] + 8, lo[2]:lo[2] + 8].cpu().numpy()
            assert np.array_equal(got, ref), (dil, lo)
        del y


@pytest.mark.parametrize("dtype,rad", [(np.uint8, 7), (np.uint16, 9), (np.float16, 12),
                                       (np.float32, 16), (np.uint16, 16)])
def test_cube_large_radius_van_herk(dtype, rad):
    """Cube radii above the tiled kernels run three van Herk / Gil-Werman
    line passes: bit-exact against the oracle's brute force, on a volume
    with ragged line tiles (130 = 128 + 2 outputs along x, 33 lines of a
    32-line tile) and extents shorter than the window (every sample
    reflected several times). Small volumes: the oracle visits (2r + 1)^3
    sources per voxel."""
    for shape in [(4, 33, 130), (5, 11, 9)]:
        f = rand_volume(dtype, shape, 30 + rad)
        x = to_dev(f)
        e = to_np(hp.erode3d(x, "cube", rad))
        d = to_np(hp.dilate3d(x, "cube", rad))
        assert np.array_equal(e.view(np.uint8), oracle.erode3d(f, oracle.SE_CUBE, rad).view(np.uint8))
        assert np.array_equal(d.view(np.uint8), oracle.dilate3d(f, oracle.SE_CUBE, rad).view(np.uint8))


@pytest.mark.parametrize("rad", [2, 4])
def test_cube_thin_volume_van_herk(rad):
    """Volumes thinner than the radius in y skip the tiled kernels; the cube
    takes the line passes there as well."""
    f = rand_volume(np.float32, (12, rad - 1 if rad > 2 else 1, 50), 40 + rad)
    x = to_dev(f)
    assert np.array_equal(to_np(hp.erode3d(x, "cube", rad)), oracle.erode3d(f, oracle.SE_CUBE, rad))
    assert np.array_equal(to_np(hp.dilate3d(x, "cube", rad)), oracle.dilate3d(f, oracle.SE_CUBE, rad))


def test_cube_van_herk_out_of_core_within_budget():
    f = synth.porous((80, 96, 112), 33)[0]
    budget = 12_000_000
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(budget)
        host = hp.erode3d(f, "cube", 9)
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4 and 0 < st["peak_device_bytes"] <= budget and st["live_device_bytes"] == 0
    assert np.array_equal(host, to_np(hp.erode3d(to_dev(f), "cube", 9)))
    # the oracle on sampled boxes (corners, faces, interior), from the input box with halo
    r, b = 9, 8
    for lo in [(0, 0, 0), (72, 88, 104), (36, 0, 50), (10, 45, 0), (60, 20, 99)]:
        ilo = [max(0, c - r) for c in lo]
        ihi = [min(n, c + b + r) for c, n in zip(lo, f.shape)]
        ref = oracle.erode3d(f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]], oracle.SE_CUBE, r,
                             gdims=f.shape, in_lo=ilo, out_lo=lo, out_shape=(b, b, b))
        assert np.array_equal(host[lo[0]:lo[0] + b, lo[1]:lo[1] + b, lo[2]:lo[2] + b], ref), lo


def test_full_size_face_planes_ball3_1024():
    """Erosion and dilation (ball r = 3) of the 1024^3 step on whole face
    planes, an interior 64^3 block and an interior block across z = 256 and
    z = 288 (where z chunks of 128 or 96 planes meet), bit for bit against
    the oracle."""
    n = 1024
    f, _ = synth.porous(n, synth.SEED_BASE + 1)
    x = to_dev(f)
    rad = 3
    boxes = [((0, 0, 0), (1, n, n)), ((n - 1, 0, 0), (1, n, n)), ((0, 0, n - 1), (n, n, 1)),
             ((0, 0, 0), (n, 1, n)), ((200, 600, 900), (64, 64, 64)), ((250, 300, 400), (48, 48, 48))]
    oracle.use_threads(True)
    try:
        for fn, dil in ((hp.erode3d, False), (hp.dilate3d, True)):
            y = fn(x, "ball", rad)
            torch.cuda.synchronize()
            for lo, shp in boxes:
                ilo = [max(0, c - rad) for c in lo]
                ihi = [min(n, c + s + rad) for c, s in zip(lo, shp)]
                part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
                ref = oracle.morph3d(part, oracle.SE_BALL, rad, dil, gdims=f.shape, in_lo=ilo,
                                     out_lo=lo, out_shape=shp)
                got = y[lo[0]:lo[0] + shp[0], lo[1]:lo[1] + shp[1], lo[2]:lo[2] + shp[2]]
                assert np.array_equal(got.cpu().numpy(), ref), (dil, lo, shp)
            del y
    finally:
        oracle.use_threads(False)


@pytest.mark.parametrize("dtype,rad", [(np.uint8, 7), (np.uint16, 8), (np.float16, 9),
                                       (np.float32, 10), (np.uint16, 10)])
def test_ball_radius_7_to_10_tiled(dtype, rad):
    """Balls of radius 7-10 run the tiled z-march (x-line levels in shared
    memory, disks per |dz|, register z ring): bit-exact against the oracle
    on ragged tiles (70 = 2 x 32 + 6 columns, 36 = 32 + 4 rows) and a volume
    as thin as the radius allows."""
    for shape in [(8, 36, 70), (5, rad, rad + 1)]:
        f = rand_volume(dtype, shape, 50 + rad)
        x = to_dev(f)
        e = to_np(hp.erode3d(x, "ball", rad))
        d = to_np(hp.dilate3d(x, "ball", rad))
        assert np.array_equal(e.view(np.uint8), oracle.erode3d(f, oracle.SE_BALL, rad).view(np.uint8))
        assert np.array_equal(d.view(np.uint8), oracle.dilate3d(f, oracle.SE_BALL, rad).view(np.uint8))


@pytest.mark.parametrize("dtype,rad", [(np.uint8, 11), (np.float32, 12), (np.uint16, 13),
                                       (np.float16, 14), (np.float32, 16), (np.uint16, 16)])
def test_ball_radius_11_to_16_tiled(dtype, rad):
    """Balls of radius 11-16 run the tiled z-march on 16-row tiles (two
    output rows per thread, one line-minimum buffer, a shift ring in z):
    bit-exact against the oracle's brute force on ragged tiles (20 = 16 + 4
    rows, 40 = 32 + 8 columns), a volume as thin as the radius allows, and
    (r = 12) a z extent split into chunks of 32 and 8 planes."""
    shapes = [(8, 20, 40), (6, rad, rad + 1)] + ([(40, 20, 40)] if rad == 12 else [])
    for shape in shapes:
        f = rand_volume(dtype, shape, 70 + rad)
        x = to_dev(f)
        e = to_np(hp.erode3d(x, "ball", rad))
        d = to_np(hp.dilate3d(x, "ball", rad))
        assert np.array_equal(e.view(np.uint8), oracle.erode3d(f, oracle.SE_BALL, rad).view(np.uint8)), shape
        assert np.array_equal(d.view(np.uint8), oracle.dilate3d(f, oracle.SE_BALL, rad).view(np.uint8)), shape


def test_large_ball_out_of_core_within_budget():
    """Host-mode dilation with the r = 13 ball under a budget that forces
    several bricks: equal bit for bit to the device-mode call, within the
    budget, and equal to the oracle on sampled boxes (corners, faces,
    interior)."""
    f = synth.porous((64, 72, 80), 35)[0]
    r, b = 13, 8
    budget = 2_400_000
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(budget)
        host = hp.dilate3d(f, "ball", r)
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 3 and 0 < st["peak_device_bytes"] <= budget and st["live_device_bytes"] == 0
    assert np.array_equal(host, to_np(hp.dilate3d(to_dev(f), "ball", r)))
    for lo in [(0, 0, 0), (56, 64, 72), (30, 0, 40), (5, 40, 0), (44, 17, 71)]:
        ilo = [max(0, c - r) for c in lo]
        ihi = [min(n, c + b + r) for c, n in zip(lo, f.shape)]
        ref = oracle.dilate3d(f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]], oracle.SE_BALL, r,
                              gdims=f.shape, in_lo=ilo, out_lo=lo, out_shape=(b, b, b))
        assert np.array_equal(host[lo[0]:lo[0] + b, lo[1]:lo[1] + b, lo[2]:lo[2] + b], ref), lo
