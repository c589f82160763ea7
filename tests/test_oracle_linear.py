"""Pins for the oracle's Gaussian / derivative filters and their adjoints.

Each check compares the oracle with something other than itself: scipy.ndimage
(an independent library, same conventions: reflect = half-sample symmetric,
radius floor(truncate*sigma + 0.5), derivatives of the normalised sampled
Gaussian), closed forms, invariants, or brute force on tiny volumes with the
reflection done by numpy's 'symmetric' padding.
"""
import itertools

import numpy as np
import pytest
import scipy.ndimage as nd

import oracle
import synth

SIGMAS = [0.7, 1.0, 2.0, 3.0, 4.0]


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _taps(sigma, order, truncate=3.0):
    """Normalised sampled Gaussian and its analytic derivative, computed here."""
    r = int(np.floor(truncate * sigma + 0.5))
    k = np.arange(-r, r + 1, dtype=np.float64)
    g0 = np.exp(-0.5 * k * k / sigma**2)
    g0 /= g0.sum()
    if order == 0:
        return k, g0
    if order == 1:
        return k, -k / sigma**2 * g0
    return k, (k * k / sigma**4 - 1 / sigma**2) * g0


def test_radius_rule():
    # r = floor(3 sigma + 0.5): 0.7->2, 1->3, 2->6, 3->9, 4->12
    assert [oracle.radius(s) for s in SIGMAS] == [2, 3, 6, 9, 12]


def test_reflect_matches_numpy_symmetric_pad():
    for n in [1, 2, 3, 5]:
        pad = 13
        ext = np.pad(np.arange(n), pad, mode="symmetric")
        got = [oracle.reflect(i, n) for i in range(-pad, n + pad)]
        assert got == list(ext)


@pytest.mark.parametrize("sigma", SIGMAS)
def test_kernel_moments(sigma):
    g0, g1, g2 = (oracle.kernel1d(sigma, o) for o in (0, 1, 2))
    r = oracle.radius(sigma)
    k = np.arange(-r, r + 1)
    assert abs(g0.sum() - 1) < 1e-15
    assert np.allclose(g0, g0[::-1], rtol=0, atol=0)       # even
    assert np.allclose(g1, -g1[::-1], rtol=0, atol=0)      # odd
    assert np.allclose(g2, g2[::-1], rtol=0, atol=0)       # even
    # g1 = -k/sigma^2 g0 and g2 = (k^2/sigma^4 - 1/sigma^2) g0
    assert np.allclose(g1, -k / sigma**2 * g0, rtol=1e-14, atol=0)
    assert np.allclose(g2, (k * k / sigma**4 - 1 / sigma**2) * g0, rtol=1e-13, atol=1e-18)
    # convolution with g1 of a rising ramp is positive: sum_k g1(k)(i-k) > 0
    assert -(k * g1).sum() > 0


@pytest.mark.parametrize("sigma", SIGMAS)
@pytest.mark.parametrize("order", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0),
                                   (0, 2, 0), (0, 0, 2), (1, 1, 0), (0, 1, 2)])
def test_vs_scipy_gaussian_filter(sigma, order):
    f = _rand((11, 14, 17), 7)
    a = oracle.gaussian3d(f, sigma, order)
    b = nd.gaussian_filter(f, sigma, order=order, mode="reflect", truncate=3.0)
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
def test_input_dtypes_vs_scipy(dtype):
    rng = np.random.default_rng(3)
    if dtype in (np.uint8, np.uint16):
        f = rng.integers(0, np.iinfo(dtype).max, (9, 10, 12)).astype(dtype)
    else:
        f = rng.standard_normal((9, 10, 12)).astype(dtype)
    a = oracle.gaussian3d(f, 1.0, (0, 1, 0))
    b = nd.gaussian_filter(f.astype(np.float64), 1.0, order=(0, 1, 0), mode="reflect",
                           truncate=3.0)
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (3, 5, 8), (5, 2, 3), (8, 8, 8)])
@pytest.mark.parametrize("sigma", [0.7, 1.0, 2.0])
def test_brute_force_3d_sum(shape, sigma):
    """Direct triple sum over the tensor-product kernel, reflect via np.pad,
    on tiny volumes including r >= n."""
    f = _rand(shape, 11)
    order = (1, 0, 2)
    r = oracle.radius(sigma)
    taps = [_taps(sigma, o)[1] for o in order]
    ext = np.pad(f, r, mode="symmetric")
    ref = np.zeros(shape)
    for (iz, kz), (iy, ky), (ix, kx) in itertools.product(*[list(enumerate(range(-r, r + 1)))] * 3):
        w = taps[0][iz] * taps[1][iy] * taps[2][ix]
        # out[p] += w * f[R(p - k)]  ->  slice of the padded array
        ref += w * ext[r - kz:r - kz + shape[0], r - ky:r - ky + shape[1], r - kx:r - kx + shape[2]]
    got = oracle.gaussian3d(f, sigma, order)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("sigma", SIGMAS)
def test_constant_volume(sigma):
    c = 3.25
    f = np.full((7, 9, 30), c)
    assert np.abs(oracle.gaussian3d(f, sigma) - c).max() < 1e-13
    assert np.abs(oracle.gaussian3d(f, sigma, (0, 0, 1))).max() < 1e-13
    # LoG of a constant is 3 c sum_k g2(k) (derivatives are not re-normalised)
    _, g2 = _taps(sigma, 2)
    lap = oracle.filterbank3d(f, [(oracle.LOG, sigma)])[0]
    assert np.abs(lap - 3 * c * g2.sum()).max() < 1e-13


@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_impulse_response_is_sampled_kernel(sigma):
    r = oracle.radius(sigma)
    n = 2 * r + 9
    f = np.zeros((n, n, n))
    c = n // 2
    f[c, c, c] = 1.0
    out = oracle.gaussian3d(f, sigma)
    _, g0 = _taps(sigma, 0)
    ref = np.zeros_like(f)
    ref[c - r:c + r + 1, c - r:c + r + 1, c - r:c + r + 1] = np.einsum("i,j,k->ijk", g0, g0, g0)
    assert np.abs(out - ref).max() < 1e-16


@pytest.mark.parametrize("sigma", SIGMAS)
def test_ramp_first_derivative_closed_form(sigma):
    """f = x: interior D_x = sum_k k^2 g0(k) / sigma^2."""
    r = oracle.radius(sigma)
    nx = 2 * r + 6
    f = np.broadcast_to(np.arange(nx, dtype=np.float64), (3, 4, nx)).copy()
    dx = oracle.gaussian3d(f, sigma, (0, 0, 1))
    k, g0 = _taps(sigma, 0)
    expect = (k * k * g0).sum() / sigma**2
    assert np.abs(dx[:, :, r:nx - r] - expect).max() < 1e-12
    # and along z nothing changes
    assert np.abs(oracle.gaussian3d(f, sigma, (1, 0, 0))).max() < 1e-12


@pytest.mark.parametrize("sigma", [0.7, 2.0, 4.0])
def test_gm_and_log_vs_scipy(sigma):
    f = _rand((13, 12, 15), 5)
    gm, lap, g = oracle.filterbank3d(f, [(oracle.GM, sigma), (oracle.LOG, sigma), (oracle.G, sigma)])
    kw = dict(mode="reflect", truncate=3.0)
    assert np.abs(gm - nd.gaussian_gradient_magnitude(f, sigma, **kw)).max() < 1e-12
    assert np.abs(lap - nd.gaussian_laplace(f, sigma, **kw)).max() < 1e-12
    assert np.abs(g - nd.gaussian_filter(f, sigma, **kw)).max() < 1e-12


def test_chunked_boxes_equal_whole_volume():
    """The Z-chunked model with halos reproduces the whole-volume result."""
    f = synth.porous((40, 21, 19), 9)[0]
    sigma, order = 2.0, (0, 1, 1)
    r = oracle.radius(sigma)
    whole = oracle.gaussian3d(f, sigma, order)
    nz = f.shape[0]
    for z0, z1 in [(0, 7), (7, 20), (20, 33), (33, 40)]:
        lo, hi = max(0, z0 - r), min(nz, z1 + r)
        # faces need the reflected planes, which lie inside [0, r) / [nz-r, nz)
        part = oracle.gaussian3d(f[lo:hi], sigma, order, gdims=f.shape, in_lo=(lo, 0, 0),
                                 out_lo=(z0, 0, 0), out_shape=(z1 - z0,) + f.shape[1:])
        assert np.array_equal(part, whole[z0:z1])
    with pytest.raises(oracle.OracleError, match="halo"):
        oracle.gaussian3d(f[10:20], sigma, order, gdims=f.shape, in_lo=(10, 0, 0),
                          out_lo=(12, 0, 0), out_shape=(4,) + f.shape[1:])


# ------------------------------------------------------------------ adjoints

@pytest.mark.parametrize("sigma,order", [(1.0, (0, 0, 0)), (0.7, (1, 0, 2)), (2.0, (0, 1, 0)),
                                         (4.0, (2, 0, 1))])
def test_adjoint_dot_product(sigma, order):
    shape = (9, 13, 6)   # includes r >= n along x for sigma = 2, 4
    x = _rand(shape, 1)
    y = _rand(shape, 2)
    lhs = (oracle.gaussian3d(x, sigma, order) * y).sum()
    rhs = (x * oracle.gaussian3d_adjoint(y, sigma, order)).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_adjoint_is_dense_transpose():
    shape = (3, 4, 5)
    n = int(np.prod(shape))
    sigma, order = 1.0, (0, 1, 1)
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1
        A[:, j] = oracle.gaussian3d(e.reshape(shape), sigma, order).ravel()
    AT = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1
        AT[:, j] = oracle.gaussian3d_adjoint(e.reshape(shape), sigma, order).ravel()
    assert np.abs(A.T - AT).max() < 1e-15


def test_filterbank_vjp_finite_differences():
    """Central differences (h = 1e-3) of the FP64 forward, summed only over
    the outputs the perturbed voxel reaches."""
    shape = (12, 11, 10)
    f = synth.spheres(shape, 3, 5).astype(np.float64)
    filters = [(oracle.G, 1.0), (oracle.GM, 1.0), (oracle.LOG, 0.7), (oracle.GM, 2.0)]
    ws = [synth.normal_field(shape, 100 + i, np.float64) for i in range(len(filters))]
    g = oracle.filterbank3d_vjp(f, filters, ws)
    h = 1e-3
    rng = np.random.default_rng(0)
    for _ in range(12):
        q = tuple(int(rng.integers(0, s)) for s in shape)
        fp, fm = f.copy(), f.copy()
        fp[q] += h
        fm[q] -= h
        op = oracle.filterbank3d(fp, filters)
        om = oracle.filterbank3d(fm, filters)
        fd = sum(((a - b) * w).sum() for a, b, w in zip(op, om, ws)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1.0, abs(g[q]))


def test_filterbank_vjp_linear_parts_equal_adjoint_sum():
    shape = (7, 8, 9)
    f = _rand(shape, 4)
    w = _rand(shape, 5)
    g = oracle.filterbank3d_vjp(f, [(oracle.LOG, 1.0)], [w])
    ref = sum(oracle.gaussian3d_adjoint(w, 1.0, o) for o in [(2, 0, 0), (0, 2, 0), (0, 0, 2)])
    assert np.abs(g - ref).max() < 1e-14


def test_unsharp_mask_pins():
    """Unsharp mask: amount 0 gives the input exactly, a constant volume stays
    constant, and the definition against scipy's Gaussian (an independent
    library) for the FP64 oracle."""
    import scipy.ndimage as nd
    rng = np.random.default_rng(12)
    f = rng.standard_normal((9, 10, 11))
    assert np.array_equal(oracle.unsharp3d(f, 1.3, 0.0), f)
    c = np.full((7, 8, 9), 3.25)
    assert np.allclose(oracle.unsharp3d(c, 2.0, 1.7), c, rtol=0, atol=1e-12)
    for sigma, amount in ((1.0, 0.5), (2.0, 1.5)):
        g = nd.gaussian_filter(f, sigma, mode="reflect", truncate=3.0)
        ref = f + amount * (f - g)
        assert np.allclose(oracle.unsharp3d(f, sigma, amount), ref, rtol=0, atol=1e-12)


def test_local_threshold_pins():
    """Gaussian local threshold: on a constant volume T = c - offset, so the
    decision is offset > 0 everywhere; against scipy's Gaussian elsewhere."""
    import scipy.ndimage as nd
    c = np.full((6, 7, 8), 100.0)
    assert oracle.threshold_local(c, 1.5, 2.0)[0].all()
    assert not oracle.threshold_local(c, 1.5, -2.0)[0].any()
    rng = np.random.default_rng(4)
    f = rng.standard_normal((9, 10, 11))
    u, t = oracle.threshold_local(f, 2.0, 0.1)
    ref = nd.gaussian_filter(f, 2.0, mode="reflect", truncate=3.0) - 0.1
    assert np.allclose(t, ref, rtol=0, atol=1e-12)
    sure = np.abs(f - ref) > 1e-9
    assert np.array_equal(u[sure], (f > ref)[sure].astype(np.uint8))
