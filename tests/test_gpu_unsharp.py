"""GPU parity of the unsharp mask (Gaussian plus an FP32 epilogue) against
the FP64 oracle: max |err| <= 1e-4 x range, for every input dtype, two
sigmas and two amounts, on ragged volumes; host volumes are refused."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("sigma,amount", [(1.0, 0.5), (2.0, 1.5)])
def test_unsharp_parity(dtype, sigma, amount):
    for shape in [(13, 37, 72), (6, 20, 40)]:
        f = rand_volume(dtype, shape, 50)
        got = to_np(hp.unsharp3d(to_dev(f), sigma, amount))
        assert got.dtype == np.float32
        assert_filter_close(got, oracle.unsharp3d(f, sigma, amount), f"{dtype.__name__} {shape} s={sigma} a={amount}")


def test_host_volume_refused():
    with pytest.raises(hp.HPError):
        hp.unsharp3d(rand_volume(np.float32, (8, 8, 16), 1), 1.0, 1.0)
