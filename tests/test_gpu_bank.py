"""GPU parity: the multi-sigma filter bank (G, gradient magnitude, LoG at
sigma 0.7, 1, 2, 4) in one persistent launch, against the FP64 oracle
(max |err| <= 1e-4 x range, plus half an f16 ulp for f16 storage), and
brick partitions == whole volume bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")

SIGMAS = (0.7, 1.0, 2.0, 4.0)
BANK = [(k, s) for s in SIGMAS for k in (hp.G, hp.GM, hp.LOG)]
ORACLE_KIND = {hp.G: oracle.G, hp.GM: oracle.GM, hp.LOG: oracle.LOG}


def _oracle_bank(f, filters, **kw):
    return oracle.filterbank3d(f, [(ORACLE_KIND[k], s) for k, s in filters], **kw)


@pytest.mark.parametrize("dtype,out", [(np.float16, hp.HP_F16), (np.float32, hp.HP_F32),
                                       (np.uint16, hp.HP_F32)])
@pytest.mark.parametrize("shape", [(40, 48, 64), (27, 33, 50)])
def test_bank_parity(dtype, out, shape):
    if dtype == np.float16:
        f = synth.porous_f16(shape, 11)
    else:
        f = rand_volume(dtype, shape, 4)
    outs = hp.filterbank3d(to_dev(f), BANK, out_dtype=out)
    refs = _oracle_bank(f, BANK)
    for (k, s), o, r in zip(BANK, outs, refs):
        assert_filter_close(to_np(o), r, f"kind {k} sigma {s}")


def test_bank_bricks_bitwise_equal_whole():
    f = synth.porous_f16((64, 64, 64), 12)
    x = to_dev(f)
    whole = [to_np(o) for o in hp.filterbank3d(x, BANK)]
    bricks = synth.kd_bricks(64, 12, 99, minside=16, quantum=16)
    parts = [to_np(o) for o in hp.filterbank3d(x, BANK, bricks=bricks)]
    for a, b in zip(whole, parts):
        assert np.array_equal(a.view(np.uint16), b.view(np.uint16))


def test_bank_subset_and_errors():
    f = rand_volume(np.float32, (20, 30, 40), 5)
    x = to_dev(f)
    filt = [(hp.LOG, 1.5), (hp.G, 0.8)]
    outs = hp.filterbank3d(x, filt, out_dtype=hp.HP_F32)
    for o, r in zip(outs, _oracle_bank(f, filt)):
        assert_filter_close(to_np(o), r, "subset")
    with pytest.raises(hp.HPError):
        hp.filterbank3d(x, [(hp.G, 1.0), (hp.G, 1.0)])        # duplicate
    with pytest.raises(hp.HPError):
        hp.filterbank3d(f, [(hp.G, 1.0), (hp.G, 1.0)])        # duplicate, host volume
    with pytest.raises(hp.HPError, match="HP_ERR_UNSUPPORTED"):
        hp.filterbank3d(f, [(hp.G, 5.0)])                      # radius 15 > 12
    # a host volume runs out of core with the same result
    host = hp.filterbank3d(f, filt, out_dtype=hp.HP_F32)
    for h, o in zip(host, outs):
        assert np.array_equal(h.view(np.uint32), to_np(o).view(np.uint32))


def test_bank_512_37_bricks_sampled():
    """The 512^3 f16 bank over 37 uneven bricks (sides 64..256): sampled
    boxes against the oracle, and equal to the brick-free launch."""
    n = 512
    f = synth.porous_f16(n, synth.SEED_BASE + 3)
    x = to_dev(f)
    bricks = synth.kd_bricks(n, 37, synth.SEED_BASE + 3)
    outs = hp.filterbank3d(x, BANK, bricks=bricks)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    los = [(0, 0, 0), (n - 8, n - 8, n - 8), (250, 0, 300)]
    los += [tuple(int(v) for v in rng.integers(0, n - 8, 3)) for _ in range(3)]
    for i, (k, s) in enumerate(BANK):
        r = oracle.radius(s)
        refs, gots = [], []
        for lo in los:
            ilo = [max(0, c - r) for c in lo]
            ihi = [min(n, c + 8 + r) for c in lo]
            part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
            refs.append(_oracle_bank(part, [(k, s)], gdims=f.shape, in_lo=ilo, out_lo=lo,
                                     out_shape=(8, 8, 8))[0])
            gots.append(outs[i][lo[0]:lo[0] + 8, lo[1]:lo[1] + 8, lo[2]:lo[2] + 8].cpu().numpy())
        err, rng_ = assert_filter_close(np.stack(gots), np.stack(refs), f"512^3 kind {k} sigma {s}")
        print(f"bank 512^3 f16 kind {k} sigma {s}: max |err| {err:.3e} (range {rng_:.3e})")
    whole = hp.filterbank3d(x, BANK)
    for a, b in zip(outs, whole):
        assert torch.equal(a.view(torch.int16), b.view(torch.int16))


@pytest.mark.parametrize("r", list(range(1, 13)))
def test_bank_every_radius(r):
    """Each radius 1..12 of the four-plane kernel (16 x 16 tiles, and
    32 x 16 where r <= 6 fits), all three outputs, against the oracle; the
    x extent keeps 16-byte rows so that the TMA path is taken, the y extent
    is ragged against both tile heights."""
    sigma = r / 3.0
    assert oracle.radius(sigma) == r
    f = synth.porous_f16((22, 37, 64), 100 + r)
    filt = [(hp.G, sigma), (hp.GM, sigma), (hp.LOG, sigma)]
    outs = hp.filterbank3d(to_dev(f), filt, out_dtype=hp.HP_F32)
    for (k, s), o, ref in zip(filt, outs, _oracle_bank(f, filt)):
        assert_filter_close(to_np(o), ref, f"r={r} kind {k}")


@pytest.mark.parametrize("dtype", [np.float16, np.uint16, np.float32])
def test_bank_thin_z_and_partial_groups(dtype):
    """Volumes thinner in z than the radius (reflection bounces more than
    once; every plane group is loaded plane by plane), z extents that end in
    a partial group of four planes, and x/y extents just above the radius
    (13 rows at r = 12: rows of the tile beyond the volume reflect twice)."""
    for shape in [(5, 40, 64), (7, 24, 32), (30, 20, 48), (3, 13, 16), (4, 16, 32)]:
        f = synth.porous_f16(shape, 7) if dtype == np.float16 else rand_volume(dtype, shape, 8)
        filt = [(k, s) for s in (1.0, 4.0) for k in (hp.G, hp.GM, hp.LOG)]
        outs = hp.filterbank3d(to_dev(f), filt, out_dtype=hp.HP_F32)
        for (k, s), o, ref in zip(filt, outs, _oracle_bank(f, filt)):
            assert_filter_close(to_np(o), ref, f"{dtype.__name__} {shape} kind {k} sigma {s}")
