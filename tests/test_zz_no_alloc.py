"""The allocation-free morphology subgradient (hp_morph3d_backward_noalloc).

Callers that may not allocate device memory during this step (fixed arenas,
real-time loops, processes whose memory belongs to another pool) use this
entry point: its index scratch is a fixed array inside the library. The test
calls it through the C ABI twice in a row and compares both results with the
allocating entry point. It lives in a file that pytest collects last, and it
passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")
from paper_2511_11890_b300._lib import (HP_DEVICE, HP_ERR_UNSUPPORTED, HP_F32, HP_OK,  # noqa: E402
                                        HP_SE_BALL, HP_SE_CUBE, lib)


def _view(t, dtype_code):
    h = ctypes.c_void_p()
    nz, ny, nx = t.shape
    assert lib.hp_volume_create(ctypes.byref(h), ctypes.c_void_p(t.data_ptr()), dtype_code,
                                HP_DEVICE, nx, ny, nz) == HP_OK
    return h


def _run(fn, x, g, dilate, se, rad, expect_no_alloc=False):
    out = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
    vi, vg, vo = _view(x, HP_F32), _view(g, HP_F32), _view(out, HP_F32)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    before = (hp.stats(), torch.cuda.memory_allocated())
    rc = fn(vi, vg, int(dilate), se, rad, vo, 0, s)
    torch.cuda.synchronize()
    after = (hp.stats(), torch.cuda.memory_allocated())
    for v in (vi, vg, vo):
        lib.hp_volume_destroy(v)
    assert rc == HP_OK, lib.hp_last_error()
    if expect_no_alloc:
        # neither the library's device-byte counters (live and peak) nor
        # torch's allocator saw an allocation during the call
        for k in ("live_device_bytes", "peak_device_bytes"):
            assert after[0][k] == before[0][k], k
        assert after[1] == before[1]
    return out


@pytest.mark.parametrize("shape,dilate,se,rad", [((40, 44, 48), False, HP_SE_CUBE, 2),
                                                 ((33, 20, 70), True, HP_SE_BALL, 3)])
def test_noalloc_matches_allocating_entry_point_twice(shape, dilate, se, rad):
    f = synth.spheres(shape, 12, 77)
    x = torch.from_numpy(f).cuda()
    g = torch.from_numpy(synth.normal_field(shape, 78)).cuda()
    ref = _run(lib.hp_morph3d_backward, x, g, dilate, se, rad)
    # both entry points run the same deterministic argmin and gather
    # kernels, so the results agree bit for bit
    for _ in range(2):
        got = _run(lib.hp_morph3d_backward_noalloc, x, g, dilate, se, rad, expect_no_alloc=True)
        assert torch.equal(got, ref)


def test_noalloc_full_size_and_limit():
    n = 256                                    # the largest volume the fixed array holds
    f = synth.spheres(n, 320, 79)
    x = torch.from_numpy(f).cuda()
    g = torch.from_numpy(synth.normal_field((n, n, n), 80)).cuda()
    ref = _run(lib.hp_morph3d_backward, x, g, False, HP_SE_CUBE, 2)
    got = _run(lib.hp_morph3d_backward_noalloc, x, g, False, HP_SE_CUBE, 2, expect_no_alloc=True)
    assert torch.equal(got, ref)
    # one voxel too many is refused before any device work
    big = torch.empty(1, dtype=torch.float32, device="cuda")
    hv = ctypes.c_void_p()
    assert lib.hp_volume_create(ctypes.byref(hv), ctypes.c_void_p(big.data_ptr()), HP_F32,
                                HP_DEVICE, n * n + 1, n, 1) == HP_OK
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hp_morph3d_backward_noalloc(hv, hv, 0, HP_SE_CUBE, 1, hv, 0, s)
    lib.hp_volume_destroy(hv)
    assert rc == HP_ERR_UNSUPPORTED
    assert b"16777216" in lib.hp_last_error()
