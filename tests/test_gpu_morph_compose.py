"""GPU parity of opening, closing and white top-hat (compositions of the
erosion and dilation kernels through a scratch volume) against the oracle,
bit for bit, for every dtype, both structuring elements and radii 1..3 on
ragged volumes; host volumes are refused."""
import numpy as np
import pytest

import oracle
from gpu_util import rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SE = {"cube": oracle.SE_CUBE, "ball": oracle.SE_BALL}


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("se", ["cube", "ball"])
@pytest.mark.parametrize("rad", [1, 2, 3])
def test_compose_bitwise(dtype, se, rad):
    for shape in [(13, 37, 72), (6, 20, 40)]:
        f = rand_volume(dtype, shape, 30 + rad)
        x = to_dev(f)
        for name, fn in (("open", hp.open3d), ("close", hp.close3d), ("tophat", hp.tophat3d)):
            got = to_np(fn(x, se, rad))
            ref = getattr(oracle, name + "3d")(f, SE[se], rad)
            assert got.dtype == ref.dtype
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), (name, dtype, se, rad, shape)


def test_host_volume_refused():
    f = rand_volume(np.uint16, (8, 8, 16), 1)
    with pytest.raises(hp.HPError):
        hp.open3d(f, "ball", 1)
