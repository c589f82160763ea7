"""The memory budget holds on every path (Sec. III-D steps 1-2): Gaussians
with radii above the tiled kernels' limit (sigma 5 -> r = 15, sigma 7 ->
r = 21) run a generic three-pass path whose two FP32 scratch volumes are
part of each brick's planned stage. Out of core under a budget that forces
at least four bricks, the library's peak device bytes stay within it,
nothing is left after the call, and the result equals the in-HBM result
bit for bit (and the oracle within the filter tolerance)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_filter_close

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

BUDGET = 40_000_000


@pytest.mark.parametrize("sigma", [5.0, 7.0])
def test_large_radius_out_of_core_within_budget(sigma):
    f = synth.porous((96, 128, 160), 31)[0]
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(BUDGET)
        out = hp.gaussian3d(f, sigma)              # host volume: out of core
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4, st
    assert 0 < st["peak_device_bytes"] <= BUDGET, st
    assert st["live_device_bytes"] == 0
    dev = hp.gaussian3d(torch.from_numpy(f).cuda(), sigma).cpu().numpy()
    assert np.array_equal(out.view(np.uint32), dev.view(np.uint32))
    ref = oracle.gaussian3d(f, sigma)
    assert_filter_close(out, ref, f"sigma {sigma} out of core")


def test_large_radius_device_scratch_is_counted_and_released():
    f = synth.porous((40, 48, 64), 32)[0]
    x = torch.from_numpy(f).cuda()
    hp.gaussian3d(x, 5.0)
    torch.cuda.synchronize()
    st = hp.stats()
    # two FP32 scratch volumes of the whole volume while the call ran
    assert st["peak_device_bytes"] >= 2 * 4 * f.size
    assert st["live_device_bytes"] == 0
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(4 * f.size)           # less than the scratch
        with pytest.raises(hp.HPError, match="HP_ERR_BUDGET"):
            hp.gaussian3d(x, 5.0)
    finally:
        hp.set_memory_budget(old)
