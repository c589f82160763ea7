"""GPU parity of the Gaussian local threshold against the oracle. The
decision f > G_sigma f - offset is taken in FP32 on the GPU and in FP64 in
the oracle; the GPU's local mean is within 1e-4 x range(f) of the FP64 one
(the Gaussian parity bar), so every voxel whose FP64 margin |f - T| exceeds
that bound must get the same decision, and voxels inside it may get
either."""
import numpy as np
import pytest

import oracle
from gpu_util import rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("sigma,offset", [(1.0, 0.0), (2.0, 3.0)])
def test_local_threshold_parity(dtype, sigma, offset):
    for shape in [(13, 37, 72), (6, 20, 40)]:
        f = rand_volume(dtype, shape, 60)
        got = to_np(hp.threshold_local3d(to_dev(f), sigma, offset))
        assert got.dtype == np.uint8
        ref, t = oracle.threshold_local(f, sigma, offset)
        fr = f.astype(np.float64)
        bound = 1e-4 * (fr.max() - fr.min()) + 1e-6 * np.abs(t)
        sure = np.abs(fr - t) > bound
        assert sure.mean() > 0.9
        assert np.array_equal(got[sure], ref[sure]), (dtype, shape, sigma, offset)


def test_host_volume_refused():
    with pytest.raises(hp.HPError):
        hp.threshold_local3d(rand_volume(np.float32, (8, 8, 16), 1), 1.0, 0.0)
