"""GPU parity of the register z-march Gaussian (k_gauss_zr) at every radius
it takes (1..12), for each input type it takes (uint16, float16, float32) and
both output types, against the FP64 oracle (max |err| <= 1e-4 x range; plus
half an f16 ulp for f16 outputs).

The shapes give 16-byte row pitches for every input type (so the TMA path is
taken) and exercise ragged x/y tiles, tiles covering both faces of a small
volume (more reflected cells than the per-thread register list holds), and
z extents that end in a partial group of four planes."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SHAPES = [(21, 37, 72), (7, 11, 24), (6, 70, 40)]


def _sigma_for(r):
    # radius = floor(3 sigma + 0.5) = r
    return r / 3.0


@pytest.mark.parametrize("r", list(range(1, 13)))
@pytest.mark.parametrize("dtype", [np.uint16, np.float16, np.float32])
def test_every_radius_and_input_type(r, dtype):
    sigma = _sigma_for(r)
    assert oracle.radius(sigma) == r
    for i, shape in enumerate(SHAPES):
        f = rand_volume(dtype, shape, 10 * r + i)
        order = (0, 0, 0) if i != 1 else (1, 0, 2)
        got = to_np(hp.gaussian3d(to_dev(f), sigma, order))
        ref = oracle.gaussian3d(f, sigma, order)
        assert_filter_close(got, ref, f"{dtype.__name__} {shape} r={r} o={order}")


@pytest.mark.parametrize("r", [1, 3, 6, 9, 12])
def test_f16_output_every_tile_shape(r):
    sigma = _sigma_for(r)
    for i, shape in enumerate(SHAPES):
        f = rand_volume(np.uint16, shape, 200 + r + i)
        got = to_np(hp.gaussian3d(to_dev(f), sigma, (0, 1, 0), out_dtype=hp.HP_F16))
        assert got.dtype == np.float16
        assert_filter_close(got, oracle.gaussian3d(f, sigma, (0, 1, 0)), f"f16 out {shape} r={r}")
