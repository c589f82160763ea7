"""Several filters in one chunked pass (hp_multi3d, Sec. III-D applied to a
set of filters): every output equals the single-op call bit for bit, on
device volumes and out of core, where the input crosses the host link about
once for all ops and the budget holds."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

STEP = [("gauss", 1.0), ("gauss", 2.0), ("gauss", 4.0), ("erode", "ball", 3), ("dilate", "ball", 3)]


def _single(x, q):
    if q[0] == "gauss":
        return hp.gaussian3d(x, q[1], order=q[2] if len(q) > 2 else (0, 0, 0))
    fn = hp.erode3d if q[0] == "erode" else hp.dilate3d
    return fn(x, q[1], q[2])


def _bits(a):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint16 if a.dtype.itemsize == 2 else (np.uint32 if a.dtype.itemsize == 4 else np.uint8))


@pytest.mark.parametrize("ops", [STEP, [("gauss", 1.5, (0, 1, 2)), ("erode", "cube", 9),
                                         ("gauss", 5.0), ("dilate", "cube", 2)]])
def test_multi_equals_single_calls_device_and_host(ops):
    f = synth.porous((56, 72, 96), 71)[0]
    x = to_dev(f)
    dev = hp.multi3d(x, ops)
    refs = [_single(x, q) for q in ops]
    torch.cuda.synchronize()
    for d, r in zip(dev, refs):
        assert np.array_equal(_bits(d), _bits(r))
    budget = 30_000_000
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(budget)
        host = hp.multi3d(f, ops)
        st = hp.stats()
    finally:
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4 and st["peak_device_bytes"] <= budget and st["live_device_bytes"] == 0
    for h, r in zip(host, refs):
        assert np.array_equal(_bits(h), _bits(r))
    # the input crosses the link once for all ops: well under the H2D of the
    # separate calls under the same budget
    alone = 0
    try:
        hp.set_memory_budget(budget)
        for q in ops:
            _single(f, q)
            alone += hp.stats()["h2d_bytes"]
    finally:
        hp.set_memory_budget(old)
    assert f.nbytes <= st["h2d_bytes"] <= 0.75 * alone


def test_multi_errors():
    x = torch.zeros((4, 8, 8), dtype=torch.uint16, device="cuda")
    with pytest.raises(hp.HPError):
        hp.multi3d(x, [("gauss", -1.0)])
    with pytest.raises(hp.HPError, match="HP_ERR_UNSUPPORTED"):
        hp.multi3d(x, [("erode", "ball", 1)], outs=[torch.zeros((4, 8, 8), dtype=torch.float32, device="cuda")])


def test_multi_f16_thin_volume_and_device_list():
    """float16 input with float16 Gaussian outputs, on a volume thinner than
    the radius in y (generic Gaussian path and van Herk cube passes), device
    and out of core over a two-slot device list."""
    rng = np.random.default_rng(72)
    f = (rng.standard_normal((40, 5, 64)) * 3).astype(np.float16)
    ops = [("gauss", 2.0, (0, 0, 0), hp.HP_F16), ("gauss", 1.0, (1, 0, 0)), ("erode", "cube", 6),
           ("dilate", "ball", 2)]
    x = to_dev(f)
    dev = hp.multi3d(x, ops)
    refs = [hp.gaussian3d(x, 2.0, out_dtype=hp.HP_F16), hp.gaussian3d(x, 1.0, order=(1, 0, 0)),
            hp.erode3d(x, "cube", 6), hp.dilate3d(x, "ball", 2)]
    torch.cuda.synchronize()
    for d, r in zip(dev, refs):
        assert np.array_equal(_bits(d), _bits(r))
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(2_000_000)
        hp.set_devices([0, 0])
        host = hp.multi3d(f, ops)
        st = hp.stats()
    finally:
        hp.set_devices([])
        hp.set_memory_budget(old)
    assert st["bricks"] >= 4 and st["peak_device_bytes"] <= 2_000_000
    for h, r in zip(host, refs):
        assert np.array_equal(_bits(h), _bits(r))
