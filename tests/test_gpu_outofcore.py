"""Out-of-core execution (Sec. III-D): a 2048^3 uint16 porous volume (16 GiB)
in pinned host memory, processed under hp_set_memory_budget(8e9) as
halo-padded bricks streamed through the device. Gaussian sigma = 3 (f32
output, 32 GiB) and ball-radius-5 dilation (u16): chunked output equals the
unchunked in-HBM result bit for bit, sampled boxes (corners, face centres,
boxes straddling brick boundaries, random) match the oracle, and the
library never holds more device memory than the budget."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_filter_close

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

N = 2048
BUDGET = 8_000_000_000


@pytest.fixture(scope="module")
def volume():
    f, _ = synth.porous(N, synth.SEED_BASE + 2)
    xh = torch.from_numpy(f).pin_memory()
    return f, xh


def _compare_slabs(host_out: torch.Tensor, dev_out: torch.Tensor, slab=64):
    for z0 in range(0, N, slab):
        a = host_out[z0:z0 + slab].to(dev_out.device, non_blocking=False)
        b = dev_out[z0:z0 + slab]
        if not torch.equal(a.view(torch.int16 if a.element_size() == 2 else torch.int32),
                           b.view(torch.int16 if b.element_size() == 2 else torch.int32)):
            return z0
    return None


def _sample_boxes(rng, k=12, b=16, halo=9, in_bytes=2, out_bytes=4):
    """All 8 corners, the 6 face centres, boxes straddling each brick
    boundary of the executor's plan (same budget, halo and element sizes),
    and random boxes: k of them on top of the fixed ones."""
    e, m = N - b, N // 2 - b // 2
    los = [(z, y, x) for z in (0, e) for y in (0, e) for x in (0, e)]
    los += [(0, m, m), (e, m, m), (m, 0, m), (m, e, m), (m, m, 0), (m, m, e)]
    cores, _ = hp.plan_bricks((N, N, N), halo, in_bytes, out_bytes, BUDGET)
    for c in cores:
        for ax in range(3):
            if c[3 + ax] < N:  # an interior face of this brick's core
                lo = [int(v) for v in rng.integers(0, N - b, 3)]
                lo[ax] = int(c[3 + ax]) - b // 2
                los.append(tuple(lo))
    los += [tuple(int(v) for v in rng.integers(0, N - b, 3)) for _ in range(k)]
    return list(dict.fromkeys(los))


def _run_budgeted(fn):
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(BUDGET)
        fn()
        return hp.stats()
    finally:
        hp.set_memory_budget(old)


def test_gaussian_sigma3_out_of_core(volume):
    f, xh = volume
    out_h = torch.empty((N, N, N), dtype=torch.float32).pin_memory()
    st = _run_budgeted(lambda: hp.gaussian3d(xh, 3.0, out=out_h))
    assert st["bricks"] >= 8
    assert st["peak_device_bytes"] <= BUDGET
    assert st["live_device_bytes"] == 0
    assert st["h2d_bytes"] >= f.nbytes and st["d2h_bytes"] == out_h.numel() * 4
    # unchunked in HBM, compared slab by slab, bit for bit
    xd = xh.to("cuda")
    gd = hp.gaussian3d(xd, 3.0)
    torch.cuda.synchronize()
    assert _compare_slabs(out_h, gd) is None
    del gd, xd
    torch.cuda.empty_cache()
    # sampled oracle boxes
    r = oracle.radius(3.0)
    refs, gots = [], []
    for lo in _sample_boxes(np.random.default_rng(2), k=12):
        ilo = [max(0, c - r) for c in lo]
        ihi = [min(N, c + 16 + r) for c in lo]
        part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
        refs.append(oracle.gaussian3d(part, 3.0, gdims=f.shape, in_lo=ilo, out_lo=lo,
                                      out_shape=(16, 16, 16)))
        gots.append(out_h[lo[0]:lo[0] + 16, lo[1]:lo[1] + 16, lo[2]:lo[2] + 16].numpy())
    assert_filter_close(np.stack(gots), np.stack(refs), "2048^3 sigma 3")


def test_dilation_ball5_out_of_core(volume):
    f, xh = volume
    out_h = torch.empty((N, N, N), dtype=torch.uint16).pin_memory()
    st = _run_budgeted(lambda: hp.dilate3d(xh, "ball", 5, out=out_h))
    assert st["bricks"] >= 8
    assert st["peak_device_bytes"] <= BUDGET
    xd = xh.to("cuda")
    dd = hp.dilate3d(xd, "ball", 5)
    torch.cuda.synchronize()
    assert _compare_slabs(out_h, dd) is None
    del dd, xd
    torch.cuda.empty_cache()
    for lo in _sample_boxes(np.random.default_rng(3), k=6, halo=5, out_bytes=2):
        ilo = [max(0, c - 5) for c in lo]
        ihi = [min(N, c + 16 + 5) for c in lo]
        part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
        ref = oracle.dilate3d(part, oracle.SE_BALL, 5, gdims=f.shape, in_lo=ilo, out_lo=lo,
                              out_shape=(16, 16, 16))
        got = out_h[lo[0]:lo[0] + 16, lo[1]:lo[1] + 16, lo[2]:lo[2] + 16].numpy()
        assert np.array_equal(got, ref), lo


def test_impossible_budget_is_an_error_not_a_crash():
    f = np.zeros((8, 300, 300), np.uint16)
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(1000)
        with pytest.raises(hp.HPError, match="HP_ERR_BUDGET"):
            hp.gaussian3d(f, 1.0)
        assert hp.stats()["live_device_bytes"] == 0
    finally:
        hp.set_memory_budget(old)
    out = hp.gaussian3d(f, 1.0)          # the next call succeeds
    assert out.shape == f.shape


@pytest.mark.parametrize("fault,code", [("alloc:0", "HP_ERR_OOM"), ("alloc:3", "HP_ERR_OOM"),
                                        ("memcpy:0", "HP_ERR_CUDA"), ("memcpy:5", "HP_ERR_CUDA"),
                                        ("budget", "HP_ERR_BUDGET")])
def test_injected_host_faults_leave_no_leak(fault, code, monkeypatch):
    """Failures made on the host (HP_FAULT): the call returns its status, frees
    every library buffer, and the next call succeeds."""
    f = synth.porous((64, 48, 40), 9)[0]
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(3 * 48 * 40 * 12 * 6)          # several bricks
        monkeypatch.setenv("HP_FAULT", fault)
        with pytest.raises(hp.HPError, match=code):
            hp.gaussian3d(f, 1.0)
        assert hp.stats()["live_device_bytes"] == 0
        monkeypatch.delenv("HP_FAULT")
        out = hp.gaussian3d(f, 1.0)
        ref = hp.gaussian3d(torch.from_numpy(f).cuda(), 1.0).cpu().numpy()
        assert np.array_equal(out, ref)
    finally:
        hp.set_memory_budget(old)
