"""Pins for the oracle's grayscale morphology, threshold and subgradient.

Checked against scipy.ndimage grey_erosion / grey_dilation (independent
library, reflect mode, symmetric footprints), lattice-point counts of the
digital ball (OEIS A000605, stored in tests/golden/ball_counts.txt),
invariants (ordering, duality, idempotence) and 1D sliding-window
compositions built from numpy's symmetric padding.
"""
import os

import numpy as np
import pytest
import scipy.ndimage as nd

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ball(r):
    z, y, x = np.mgrid[-r:r + 1, -r:r + 1, -r:r + 1]
    return (z * z + y * y + x * x) <= r * r


def _vol(dtype, shape, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.uint8:
        return rng.integers(0, 256, shape).astype(np.uint8)
    if dtype == np.uint16:
        return rng.integers(0, 65536, shape).astype(np.uint16)
    return rng.standard_normal(shape).astype(dtype)


def _ball_counts():
    out = {}
    with open(os.path.join(GOLDEN, "ball_counts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                r, c = line.split()
                out[int(r)] = int(c)
    return out


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32, np.float64])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_CUBE, 2), (oracle.SE_BALL, 3),
                                    (oracle.SE_BALL, 2)])
def test_vs_scipy(dtype, se, rad):
    f = _vol(dtype, (9, 11, 13), 1)
    fp = np.ones((2 * rad + 1,) * 3, bool) if se == oracle.SE_CUBE else _ball(rad)
    e = oracle.erode3d(f, se, rad)
    d = oracle.dilate3d(f, se, rad)
    assert e.dtype == f.dtype and d.dtype == f.dtype
    # scipy has no float16 kernels; float16 -> float32 is exact, so compare there
    fs = f.astype(np.float32) if dtype == np.float16 else f
    assert np.array_equal(e.astype(fs.dtype), nd.grey_erosion(fs, footprint=fp, mode="reflect"))
    assert np.array_equal(d.astype(fs.dtype), nd.grey_dilation(fs, footprint=fp, mode="reflect"))


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (3, 4, 2), (1, 7, 1)])
def test_tiny_shapes_radius_beyond_extent(shape):
    f = _vol(np.uint16, shape, 2)
    for se, rad in [(oracle.SE_CUBE, 2), (oracle.SE_BALL, 5)]:
        fp = np.ones((2 * rad + 1,) * 3, bool) if se == oracle.SE_CUBE else _ball(rad)
        assert np.array_equal(oracle.erode3d(f, se, rad),
                              nd.grey_erosion(f, footprint=fp, mode="reflect"))


def test_ball_lattice_counts_golden():
    counts = _ball_counts()
    for r, c in counts.items():
        assert _ball(r).sum() == c
        n = 2 * r + 5
        f = np.zeros((n, n, n), np.uint16)
        f[n // 2, n // 2, n // 2] = 1000
        d = oracle.dilate3d(f, oracle.SE_BALL, r)
        assert int((d == 1000).sum()) == c
        c0 = n // 2
        assert np.array_equal(d[c0 - r:c0 + r + 1, c0 - r:c0 + r + 1, c0 - r:c0 + r + 1] == 1000,
                              _ball(r))


@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_BALL, 3)])
def test_invariants(se, rad):
    f = synth.porous((20, 18, 16), 3)[0]
    e = oracle.erode3d(f, se, rad)
    d = oracle.dilate3d(f, se, rad)
    assert (e <= f).all() and (f <= d).all()
    # duality on u16: eps(f) = 65535 - delta(65535 - f)
    assert np.array_equal(e, 65535 - oracle.dilate3d(65535 - f, se, rad))
    # opening and closing are idempotent
    op = oracle.dilate3d(e, se, rad)
    assert np.array_equal(oracle.dilate3d(oracle.erode3d(op, se, rad), se, rad), op)
    cl = oracle.erode3d(d, se, rad)
    assert np.array_equal(oracle.erode3d(oracle.dilate3d(cl, se, rad), se, rad), cl)
    # float duality: eps(f) = -delta(-f)
    g = f.astype(np.float32) / 7
    assert np.array_equal(oracle.erode3d(g, se, rad), -oracle.dilate3d(-g, se, rad))


def _line_min(f, axis, rho):
    ext = np.pad(f, [(rho, rho) if a == axis else (0, 0) for a in range(3)], mode="symmetric")
    out = None
    n = f.shape[axis]
    for o in range(2 * rho + 1):
        sl = [slice(None)] * 3
        sl[axis] = slice(o, o + n)
        v = ext[tuple(sl)]
        out = v if out is None else np.minimum(out, v)
    return out


@pytest.mark.parametrize("rho", [1, 2, 4])
def test_cube_is_three_line_erosions(rho):
    f = _vol(np.float32, (7, 12, 10), 5)
    ref = _line_min(_line_min(_line_min(f, 2, rho), 1, rho), 0, rho)
    assert np.array_equal(oracle.erode3d(f, oracle.SE_CUBE, rho), ref)


def test_chunked_boxes_equal_whole_volume():
    f = synth.porous((30, 17, 15), 4)[0]
    rad = 3
    whole = oracle.dilate3d(f, oracle.SE_BALL, rad)
    for z0, z1 in [(0, 2), (2, 11), (11, 30)]:
        lo, hi = max(0, z0 - rad), min(30, z1 + rad)
        part = oracle.dilate3d(f[lo:hi], oracle.SE_BALL, rad, gdims=f.shape, in_lo=(lo, 0, 0),
                               out_lo=(z0, 0, 0), out_shape=(z1 - z0,) + f.shape[1:])
        assert np.array_equal(part, whole[z0:z1])


def test_threshold():
    f = np.array([0.5, np.nextafter(np.float32(0.5), np.float32(1)), 0.49, -1, 2],
                 np.float32).reshape(1, 1, 5)
    assert oracle.threshold(f, 0.5).ravel().tolist() == [0, 1, 0, 0, 1]


# --------------------------------------------------------------- subgradient

@pytest.mark.parametrize("dilate", [False, True])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 2), (oracle.SE_BALL, 2)])
def test_vjp_finite_differences_away_from_ties(dilate, se, rad):
    """FD of the FP64 forward is exact where the extreme is unique by a gap > h."""
    shape = (9, 10, 11)
    f = np.random.default_rng(8).standard_normal(shape)
    w = synth.normal_field(shape, 21, np.float64)
    g, arg = oracle.morph3d_vjp(f, se, rad, dilate, w, return_arg=True)
    h = 1e-6
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(60):
        q = tuple(int(rng.integers(0, s)) for s in shape)
        fp, fm = f.copy(), f.copy()
        fp[q] += h
        fm[q] -= h
        op = oracle.morph3d(fp, se, rad, dilate)
        om = oracle.morph3d(fm, se, rad, dilate)
        fd = ((op - om) * w).sum() / (2 * h)
        assert abs(fd - g[q]) < 1e-6 * max(1.0, abs(g[q]))
        checked += 1
    assert checked == 60
    # every routed source holds the extreme value
    m = oracle.morph3d(f, se, rad, dilate)
    assert np.array_equal(f.ravel()[arg.ravel()], m.ravel())


def test_vjp_tie_rule_constant_volume():
    """All sources tie on a constant volume: an interior voxel routes to its
    smallest-index source, which is p - (rho, rho, rho) for the cube."""
    shape = (8, 9, 10)
    rho = 2
    f = np.full(shape, 7, np.uint16)
    w = np.ones(shape)
    _, arg = oracle.morph3d_vjp(f, oracle.SE_CUBE, rho, False, w, return_arg=True)
    for p in [(3, 4, 5), (2, 2, 2), (5, 6, 7)]:
        q = np.ravel_multi_index(tuple(c - rho for c in p), shape)
        assert arg[p] == q
    # at the origin face the sources reflect onto [0, rho): smallest is 0
    assert arg[0, 0, 0] == 0
    # ball of radius 2: smallest linear index source is (z - 2, y, x)
    _, arg = oracle.morph3d_vjp(f, oracle.SE_BALL, 2, True, w, return_arg=True)
    assert arg[4, 4, 4] == np.ravel_multi_index((2, 4, 4), shape)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float32, np.float64])
@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_BALL, 2)])
def test_open_close_tophat_vs_scipy(dtype, se, rad):
    """Opening, closing and white top-hat against scipy.ndimage's own
    compositions (grey_opening, grey_closing, white_tophat, reflect mode)."""
    f = _vol(dtype, (9, 11, 13), 2)
    fp = np.ones((2 * rad + 1,) * 3, bool) if se == oracle.SE_CUBE else _ball(rad)
    assert np.array_equal(oracle.open3d(f, se, rad), nd.grey_opening(f, footprint=fp, mode="reflect"))
    assert np.array_equal(oracle.close3d(f, se, rad), nd.grey_closing(f, footprint=fp, mode="reflect"))
    assert np.array_equal(oracle.tophat3d(f, se, rad), nd.white_tophat(f, footprint=fp, mode="reflect"))


@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 2), (oracle.SE_BALL, 3)])
def test_open_close_invariants(se, rad):
    """Opening is anti-extensive and idempotent, closing extensive and
    idempotent, the top-hat non-negative and zero on a constant volume."""
    f = _vol(np.uint16, (10, 12, 14), 3)
    o, c = oracle.open3d(f, se, rad), oracle.close3d(f, se, rad)
    assert (o <= f).all() and (c >= f).all()
    assert np.array_equal(oracle.open3d(o, se, rad), o)
    assert np.array_equal(oracle.close3d(c, se, rad), c)
    t = oracle.tophat3d(f, se, rad)
    assert np.array_equal(t.astype(np.int64), f.astype(np.int64) - o.astype(np.int64))
    k = np.full((6, 7, 8), 1234, np.uint16)
    assert not oracle.tophat3d(k, se, rad).any()


# ------------------------------------------- totalOrder: signed zeros, NaN

def _f32(bits):
    return np.array(bits, np.uint32).view(np.float32).reshape(1, 1, -1)


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint16).ravel().tolist()


P0, N0 = 0x00000000, 0x80000000  # float32 +0, -0
PNAN, NNAN = 0x7FC00000, 0xFFC00000
PINF, NINF, ONE = 0x7F800000, 0xFF800000, 0x3F800000


def test_signed_zero_order_hand_built():
    """-0 < +0 in min and max: values worked out by hand on a 1 x 1 x 4
    line (cube r = 1, reflect: x = 0 reads x = 0, 0, 1; x = 3 reads 2, 3, 3)."""
    f = _f32([P0, N0, P0, P0])
    assert _bits(oracle.erode3d(f, oracle.SE_CUBE, 1)) == [N0, N0, N0, P0]
    assert _bits(oracle.dilate3d(f, oracle.SE_CUBE, 1)) == [P0, P0, P0, P0]
    w = np.array([1.0, 2.0, 4.0, 8.0]).reshape(1, 1, 4)
    # erosion: x = 0, 1, 2 route to the only -0 (x = 1); x = 3 sees +0 at
    # x = 2, 3 (tie) and takes x = 2
    g = oracle.morph3d_vjp(f, oracle.SE_CUBE, 1, False, w)
    assert g.ravel().tolist() == [0.0, 7.0, 8.0, 0.0]
    # dilation: x = 0 -> 0, x = 1 -> 0 (+0 at 0 and 2), x = 2 -> 2, x = 3 -> 2
    g = oracle.morph3d_vjp(f, oracle.SE_CUBE, 1, True, w)
    assert g.ravel().tolist() == [3.0, 0.0, 12.0, 0.0]
    # float16 and float64 follow the same order
    h = np.array([0x0000, 0x8000, 0x0000, 0x0000], np.uint16).view(np.float16).reshape(1, 1, 4)
    assert _bits(oracle.erode3d(h, oracle.SE_BALL, 1)) == [0x8000, 0x8000, 0x8000, 0x0000]
    d = np.array([0.0, -0.0, 0.0, 0.0]).reshape(1, 1, 4)
    assert np.signbit(oracle.erode3d(d, oracle.SE_CUBE, 1)).ravel().tolist() == [True, True, True, False]


def test_nan_and_inf_order_hand_built():
    """NaN with the sign bit clear is above +inf, with it set below -inf;
    line [1, +NaN, -inf, -NaN, +inf], cube r = 1, worked out by hand."""
    f = _f32([ONE, PNAN, NINF, NNAN, PINF])
    assert _bits(oracle.erode3d(f, oracle.SE_CUBE, 1)) == [ONE, NINF, NNAN, NNAN, NNAN]
    assert _bits(oracle.dilate3d(f, oracle.SE_CUBE, 1)) == [PNAN, PNAN, PNAN, PINF, PINF]
    # NaNs of one sign by significand field: ascending for +, descending for -
    f = _f32([PNAN | 1, PNAN, PNAN | 1])
    assert _bits(oracle.erode3d(f, oracle.SE_CUBE, 1)) == [PNAN, PNAN, PNAN]
    assert _bits(oracle.dilate3d(f, oracle.SE_CUBE, 1)) == [PNAN | 1] * 3
    f = _f32([NNAN | 1, NNAN, NNAN | 1])
    assert _bits(oracle.erode3d(f, oracle.SE_CUBE, 1)) == [NNAN | 1] * 3
    assert _bits(oracle.dilate3d(f, oracle.SE_CUBE, 1)) == [NNAN, NNAN, NNAN]
    h = np.array([0x3C00, 0x7E00, 0xFC00, 0xFE00, 0x7C00], np.uint16).view(np.float16).reshape(1, 1, 5)
    assert _bits(oracle.erode3d(h, oracle.SE_CUBE, 1)) == [0x3C00, 0xFC00, 0xFE00, 0xFE00, 0xFE00]
    assert _bits(oracle.dilate3d(h, oracle.SE_CUBE, 1)) == [0x7E00, 0x7E00, 0x7E00, 0x7C00, 0x7C00]
    # the subgradient routes to the source the forward copied
    w = np.ones((1, 1, 5))
    _, arg = oracle.morph3d_vjp(f.reshape(1, 1, 3), oracle.SE_CUBE, 1, False, w[..., :3], return_arg=True)
    assert arg.ravel().tolist() == [0, 0, 2]


def _f16_table():
    """Every finite float16 value (as exact Fractions) sorted, with its bits."""
    from fractions import Fraction
    bits = np.arange(65536, dtype=np.uint16)
    vals = bits.view(np.float16)
    ok = np.isfinite(vals) & ~((bits == 0x8000))
    return sorted((Fraction(float(v)), int(b)) for v, b in zip(vals[ok], bits[ok]))


def _rne_f16(x, table):
    """Round the exact rational x to float16 by brute force: nearest entry
    of the table, ties to the even significand (bit pattern LSB 0)."""
    import bisect
    keys = [t[0] for t in table]
    i = bisect.bisect_left(keys, x)
    cands = [table[j] for j in (i - 1, i) if 0 <= j < len(table)]
    best = min(cands, key=lambda t: (abs(t[0] - x), t[1] & 1))
    return best[1]


@pytest.mark.parametrize("se,rad", [(oracle.SE_CUBE, 1), (oracle.SE_BALL, 2)])
def test_tophat_f16_is_one_rounding_of_the_exact_difference(se, rad):
    """float16 top-hat: every voxel is the exact rational f - opening(f)
    rounded once to float16 by a brute-force nearest-value search."""
    from fractions import Fraction
    table = _f16_table()
    rng = np.random.default_rng(11)
    # wide exponent spread, so differences lose bits when rounded
    f = (rng.standard_normal((5, 6, 7)) * 2.0 ** rng.integers(-12, 12, (5, 6, 7))).astype(np.float16)
    o = oracle.open3d(f, se, rad)
    t = oracle.tophat3d(f, se, rad)
    got = t.view(np.uint16).ravel().tolist()
    for k, (a, b) in enumerate(zip(f.ravel(), o.ravel())):
        want = _rne_f16(Fraction(float(a)) - Fraction(float(b)), table)
        assert got[k] == want or (want == 0 and got[k] in (0, 0x8000)), (k, a, b)


def test_f16_difference_rounded_through_f32_is_rounded_once():
    """FP32 has 24 >= 2 x 11 + 2 significand bits, so rounding a float16
    difference to FP32 and then to float16 equals rounding it once: checked
    against the brute-force rounding on pairs across the exponent range."""
    from fractions import Fraction
    table = _f16_table()
    rng = np.random.default_rng(12)
    a = (rng.standard_normal(3000) * 2.0 ** rng.integers(-14, 15, 3000)).astype(np.float16)
    b = (rng.standard_normal(3000) * 2.0 ** rng.integers(-14, 15, 3000)).astype(np.float16)
    ok = np.isfinite(a.astype(np.float32) - b.astype(np.float32))
    via32 = (a.astype(np.float32) - b.astype(np.float32)).astype(np.float16)
    for x, y, v in zip(a[ok], b[ok], via32[ok]):
        ex = Fraction(float(x)) - Fraction(float(y))
        if abs(ex) > 65504:
            continue
        want = _rne_f16(ex, table)
        got = int(np.array(v).view(np.uint16))
        assert got == want or (want == 0 and got in (0, 0x8000))
