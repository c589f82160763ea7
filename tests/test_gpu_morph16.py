"""GPU parity of the packed 16-bit erosion / dilation kernels (uint16 and
float16 volumes whose rows are 16-byte multiples; the register strip kernel
for radii 1..3, the buffered one above): bit-exact against the
oracle over every radius it takes, both structuring elements, several x
tiles with a partial last tile, y extents that are not multiples of the
tile height, volumes thinner than the radius allows for a full halo, and
out-of-core bricks split along x and y."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SE_NAME = {oracle.SE_CUBE: "cube", oracle.SE_BALL: "ball"}


def _check(f, se, rad):
    x = to_dev(f)
    e = to_np(hp.erode3d(x, SE_NAME[se], rad))
    d = to_np(hp.dilate3d(x, SE_NAME[se], rad))
    assert np.array_equal(e.view(np.uint16), oracle.erode3d(f, se, rad).view(np.uint16)), "erode"
    assert np.array_equal(d.view(np.uint16), oracle.dilate3d(f, se, rad).view(np.uint16)), "dilate"


@pytest.mark.parametrize("rad", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("se", [oracle.SE_BALL, oracle.SE_CUBE])
def test_radii_u16_ragged_tiles(se, rad):
    # 136 = two full 64-wide tiles + 8; 37 rows = one full 32-row tile + 5
    f = rand_volume(np.uint16, (19, 37, 136), 10 + rad)
    _check(f, se, rad)


@pytest.mark.parametrize("rad", [1, 2, 3, 6])
@pytest.mark.parametrize("se", [oracle.SE_BALL, oracle.SE_CUBE])
def test_radii_f16(se, rad):
    f = rand_volume(np.float16, (14, 40, 72), 20 + rad)
    _check(f, se, rad)


def test_f16_special_values():
    rng = np.random.default_rng(5)
    specials = np.array([np.inf, -np.inf, 65504, -65504, 6.1e-5, -6.1e-5, 6e-8, -6e-8, 1.0, -1.0],
                        np.float16)
    f = rand_volume(np.float16, (12, 33, 64), 7)
    mask = rng.random(f.shape) < 0.2
    f[mask] = rng.choice(specials, int(mask.sum()))
    for rad in (1, 3):
        _check(f, oracle.SE_BALL, rad)
        _check(f, oracle.SE_CUBE, rad)


@pytest.mark.parametrize("shape", [(9, 6, 8), (7, 3, 16), (40, 6, 24)])
@pytest.mark.parametrize("rad", [1, 2, 3, 6])
def test_thin_volumes(shape, rad):
    # extents down to the radius itself: every tile is a face tile and the
    # reflected sources fold across the whole extent
    if min(shape[1:]) < rad:
        pytest.skip("extent below the radius takes the generic kernel")
    f = rand_volume(np.uint16, shape, 3)
    _check(f, oracle.SE_BALL, rad)
    _check(f, oracle.SE_CUBE, rad)


def test_porous_ties_and_plateaus():
    # the porous phantom has long runs of equal values (ties everywhere)
    f = synth.porous((48, 70, 96), 4)[0]
    for rad in (2, 3, 5):
        _check(f, oracle.SE_BALL, rad)


@pytest.mark.parametrize("se,rad,dil,budget", [(oracle.SE_BALL, 3, False, 60_000),
                                               (oracle.SE_BALL, 6, True, 200_000),
                                               (oracle.SE_CUBE, 4, True, 100_000)])
def test_bricks_split_in_x_and_y(se, rad, dil, budget):
    """Bricks narrower than the volume in x and y (a budget that forces x
    splits): chunked result equals the whole-volume result bit for bit."""
    f = synth.porous((16, 64, 208), 12)[0]
    cores, _ = hp.plan_bricks(f.shape, rad, 2, 2, budget)
    assert len({(c[2], c[5]) for c in cores.tolist()}) > 1, "plan has no x split"
    fn = hp.dilate3d if dil else hp.erode3d
    whole = to_np(fn(to_dev(f), SE_NAME[se], rad))
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(budget)
        out = np.empty_like(f)
        fn(f, SE_NAME[se], rad, out=out)
        assert hp.stats()["bricks"] == len(cores)
    finally:
        hp.set_memory_budget(old)
    assert np.array_equal(out, whole)
    ref = oracle.morph3d(f, se, rad, dil)
    assert np.array_equal(out, ref)
