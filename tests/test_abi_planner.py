"""CPU tests of the C ABI library: it loads, exports every declared entry
point, and its host-only chunk planner (hp_plan_bricks) is correct. The
planner's bricks are also run through the oracle: halo-padded chunks must
reproduce the whole-volume result bit for bit (Sec. III-D, overlapping
context-preserving chunks)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2511_11890_b300 as hp
    lib = ctypes.CDLL(hp.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(hp.EXPORTS) == declared


def test_version_and_budget_roundtrip():
    import paper_2511_11890_b300 as hp
    assert "sm_103a" in hp.version()
    old = hp.get_memory_budget()
    hp.set_memory_budget(123456789)
    assert hp.get_memory_budget() == 123456789
    hp.set_memory_budget(old)


def test_invalid_arguments_are_reported():
    import paper_2511_11890_b300 as hp
    from paper_2511_11890_b300._lib import lib, HP_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.hp_volume_create(ctypes.byref(h), None, 0, 0, 0, 4, 4) == HP_ERR_INVALID_ARG
    assert b"extents" in lib.hp_last_error()
    with pytest.raises(hp.HPError):
        hp.plan_bricks((10, 10, 10), 2, 2, 4, 10, 3, 1)   # budget far too small


def _hull_ok(core, box, shape, halo):
    for a in range(3):
        need = {oracle.reflect(c, shape[a]) for c in range(core[a] - halo, core[3 + a] + halo)}
        if min(need) < box[a] or max(need) >= box[3 + a]:
            return False
        if box[a] < 0 or box[3 + a] > shape[a]:
            return False
    return True


@pytest.mark.parametrize("shape,halo,budget,min_bricks", [
    ((100, 64, 64), 6, 10**6, 8),
    ((37, 29, 41), 3, 2 * 10**5, 8),
    ((9, 300, 200), 12, 4 * 10**6, 8),       # one plane + halos too big -> y split
    ((5, 8, 2000), 2, 2 * 10**4, 1),         # x split
    ((1, 1, 1), 5, 10**6, 8),
])
def test_plan_tiles_volume_and_fits_budget(shape, halo, budget, min_bricks):
    import paper_2511_11890_b300 as hp
    cores, boxes = hp.plan_bricks(shape, halo, 2, 4, budget, 3, min_bricks)
    cover = np.zeros(shape, np.int32)
    for c, b in zip(cores, boxes):
        cover[c[0]:c[3], c[1]:c[4], c[2]:c[5]] += 1
        assert _hull_ok(c, b, shape, halo)
        vin = np.prod(b[3:] - b[:3]) * 2
        vout = np.prod(c[3:] - c[:3]) * 4
        assert 3 * (vin + vout) <= budget
    assert (cover == 1).all()
    if shape[0] >= min_bricks and len(cores) > 1 and (cores[:, 4] - cores[:, 1] == shape[1]).all():
        assert len(cores) >= min(min_bricks, shape[0])


def test_planned_chunks_reproduce_whole_volume_in_the_oracle():
    f = synth.porous((48, 40, 36), 12)[0]
    sigma, order = 2.0, (1, 0, 0)
    r = oracle.radius(sigma)
    import paper_2511_11890_b300 as hp
    cores, boxes = hp.plan_bricks(f.shape, r, 2, 4, 3 * (40 * 36 * 30), 3, 8)
    assert len(cores) > 3
    whole = oracle.gaussian3d(f, sigma, order)
    out = np.full(f.shape, np.nan)
    for c, b in zip(cores, boxes):
        part = f[b[0]:b[3], b[1]:b[4], b[2]:b[5]]
        out[c[0]:c[3], c[1]:c[4], c[2]:c[5]] = oracle.gaussian3d(
            part, sigma, order, gdims=f.shape, in_lo=b[:3], out_lo=c[:3], out_shape=c[3:] - c[:3])
    assert np.array_equal(out, whole)
    # morphology through the same plan
    cores, boxes = hp.plan_bricks(f.shape, 3, 2, 2, 3 * (40 * 36 * 20), 3, 8)
    whole = oracle.dilate3d(f, oracle.SE_BALL, 3)
    out = np.zeros_like(f)
    for c, b in zip(cores, boxes):
        part = f[b[0]:b[3], b[1]:b[4], b[2]:b[5]]
        out[c[0]:c[3], c[1]:c[4], c[2]:c[5]] = oracle.dilate3d(
            part, oracle.SE_BALL, 3, gdims=f.shape, in_lo=b[:3], out_lo=c[:3],
            out_shape=c[3:] - c[:3])
    assert np.array_equal(out, whole)
