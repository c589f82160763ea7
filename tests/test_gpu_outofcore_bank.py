"""Out-of-core filter bank and multi-device placement (Sec. III-D):

- host volumes in, host volumes out: the 12-filter bank on a 512^3 float16
  porous volume under a budget that forces at least eight Z slabs equals the
  in-HBM bank bit for bit, never holds more library device memory than the
  budget, sends the input across the host link about once for all twelve
  outputs, and releases everything;
- a device list that names the same GPU twice (two placement slots, each
  with its own streams and stages, sharing that device's budget) and a brick
  shard split over two passes give the single-device result bit for bit.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SIGMAS = (0.7, 1.0, 2.0, 4.0)
BANK = [(k, s) for s in SIGMAS for k in (hp.G, hp.GM, hp.LOG)]


def _budgeted(budget, fn):
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(budget)
        out = fn()
        return out, hp.stats()
    finally:
        hp.set_memory_budget(old)


def _bits(a):
    a = a.numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint16 if a.dtype == np.float16 else np.uint32)


@pytest.mark.parametrize("pinned", [False, True])
def test_bank_512_f16_out_of_core_equals_device(pinned):
    f = synth.porous_f16(512, synth.SEED_BASE + 4)
    xh = torch.from_numpy(f)
    if pinned:
        xh = xh.pin_memory()
    budget = 1_200_000_000
    outs, st = _budgeted(budget, lambda: hp.filterbank3d(xh, BANK))
    assert st["bricks"] >= 8, st
    assert 0 < st["peak_device_bytes"] <= budget, st
    assert st["live_device_bytes"] == 0
    # input once plus the slabs' halo planes; outputs once each
    assert f.nbytes <= st["h2d_bytes"] <= 1.6 * f.nbytes, st
    assert st["d2h_bytes"] == len(BANK) * f.size * 2
    dev = hp.filterbank3d(xh.cuda(), BANK)
    torch.cuda.synchronize()
    for i, (o, d) in enumerate(zip(outs, dev)):
        assert np.array_equal(_bits(o), _bits(d.cpu())), BANK[i]


def test_bank_u16_f32_outputs_out_of_core_small_budget():
    f = synth.porous((70, 96, 128), 41)[0]
    filters = [(hp.G, 1.0), (hp.GM, 2.0), (hp.LOG, 2.0), (hp.GM, 0.7)]
    outs, st = _budgeted(30_000_000, lambda: hp.filterbank3d(f, filters, out_dtype=hp.HP_F32))
    assert st["bricks"] >= 4 and st["peak_device_bytes"] <= 30_000_000
    dev = hp.filterbank3d(torch.from_numpy(f).cuda(), filters, out_dtype=hp.HP_F32)
    for o, d in zip(outs, dev):
        assert np.array_equal(_bits(o), _bits(d.cpu()))


def test_bank_host_budget_error_and_refusals():
    f = np.zeros((8, 64, 64), np.float16)
    _, _ = None, None
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(10_000)
        with pytest.raises(hp.HPError, match="HP_ERR_BUDGET"):
            hp.filterbank3d(f, BANK)
    finally:
        hp.set_memory_budget(old)
    assert hp.stats()["live_device_bytes"] == 0
    with pytest.raises(hp.HPError, match="HP_ERR_UNSUPPORTED"):   # brick lists: device only
        hp.filterbank3d(f, BANK[:1], bricks=[[0, 0, 0, 8, 64, 64]])


@pytest.mark.parametrize("op", ["gauss", "dilate", "bank"])
def test_two_device_slots_and_two_shards_equal_one_device(op):
    f = synth.porous((60, 72, 96), 43)[0]
    budget = 24_000_000
    if op == "gauss":
        run = lambda out=None: hp.gaussian3d(f, 2.0, out=out)
    elif op == "dilate":
        run = lambda out=None: hp.dilate3d(f, "ball", 3, out=out)
    else:
        run = lambda out=None: hp.filterbank3d(f, [(hp.G, 1.0), (hp.LOG, 2.0)], outs=out,
                                               out_dtype=hp.HP_F32)
    ref, st1 = _budgeted(budget, run)
    try:
        hp.set_devices([0, 0])
        two, st2 = _budgeted(budget, run)
    finally:
        hp.set_devices([])
    assert hp.get_devices() == []
    assert st2["peak_device_bytes"] <= budget and st2["live_device_bytes"] == 0
    refs = ref if isinstance(ref, list) else [ref]
    twos = two if isinstance(two, list) else [two]
    for a, b in zip(refs, twos):
        assert np.array_equal(_bits(a), _bits(b))
    # two shards of the same call, each writing only its bricks' cores
    fill = lambda: [np.full_like(r, np.nan if r.dtype.kind == "f" else 0) for r in refs]
    parts = []
    try:
        for rank in range(2):
            hp.set_brick_shard(rank, 2)
            out = fill()
            _budgeted(budget, lambda: run(out if op == "bank" else out[0]))
            parts.append(out)
    finally:
        hp.set_brick_shard(0, 1)
    for k, r in enumerate(refs):
        a, b = parts[0][k], parts[1][k]
        if r.dtype.kind == "f":
            wa, wb = ~np.isnan(a), ~np.isnan(b)
            assert not (wa & wb).any() and (wa | wb).all()   # every voxel exactly once
            merged = np.where(wa, a, b)
        else:
            merged = np.maximum(a, b)                       # u16 dilation of values > 0
        assert np.array_equal(_bits(merged), _bits(r))


def test_shard_needs_an_explicit_budget():
    f = np.zeros((16, 16, 16), np.uint16)
    old = hp.get_memory_budget()
    try:
        hp.set_memory_budget(0)
        hp.set_brick_shard(1, 2)
        with pytest.raises(hp.HPError, match="HP_ERR_INVALID_ARG"):
            hp.gaussian3d(f, 1.0)
    finally:
        hp.set_brick_shard(0, 1)
        hp.set_memory_budget(old)
    with pytest.raises(hp.HPError):
        hp.set_brick_shard(2, 2)
    with pytest.raises(hp.HPError):
        hp.set_devices([10_000])
