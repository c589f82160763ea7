"""Pins for the oracle's Hessian features and box-window local thresholds
(Sec. III-C: "Hessian" texture features; mean, Niblack and Sauvola
threshold algorithms).

Each check compares the oracle with something other than itself: scipy's
Gaussian derivative filters (mixed orders) and uniform / generic filters,
brute-force window sums over numpy's symmetric padding, a textbook cyclic
Jacobi eigensolver written here, the trace identity with the oracle's LoG,
closed forms on constant and separable quadratic volumes.
"""
import numpy as np
import pytest
import scipy.ndimage as nd

import oracle


def _rand(shape, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    if dtype == np.uint16:
        return rng.integers(0, 65536, shape).astype(np.uint16)
    if dtype == np.uint8:
        return rng.integers(0, 256, shape).astype(np.uint8)
    return rng.standard_normal(shape).astype(dtype)


# ------------------------------------------------------------------ Hessian

@pytest.mark.parametrize("sigma", [0.7, 1.0, 2.0])
def test_hessian_components_vs_scipy(sigma):
    f = _rand((9, 10, 11), 1)
    got = oracle.hessian3d(f, sigma)
    for o, g in zip(oracle.HESSIAN_ORDERS, got):
        ref = nd.gaussian_filter(f, sigma, order=o, mode="reflect", truncate=3.0)
        assert np.allclose(g, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), o


def _jacobi_eigvals(a, sweeps=30):
    """Cyclic Jacobi rotations on a symmetric 3x3 matrix (textbook method)."""
    a = np.array(a, np.float64)
    for _ in range(sweeps):
        off = a[0, 1] ** 2 + a[0, 2] ** 2 + a[1, 2] ** 2
        if off < 1e-30 * max(1.0, np.abs(a).max() ** 2):
            break
        for p, q in ((0, 1), (0, 2), (1, 2)):
            if a[p, q] == 0.0:
                continue
            th = (a[q, q] - a[p, p]) / (2.0 * a[p, q])
            t = np.sign(th) / (abs(th) + np.sqrt(th * th + 1.0)) if th != 0 else 1.0
            c = 1.0 / np.sqrt(t * t + 1.0)
            s = t * c
            j = np.eye(3)
            j[p, p] = j[q, q] = c
            j[p, q] = s
            j[q, p] = -s
            a = j.T @ a @ j
    return np.sort(np.diag(a))


def test_hessian_eigenvalues_vs_jacobi_and_trace():
    f = _rand((8, 9, 10), 2)
    sigma = 1.0
    ev = oracle.hessian_eigenvalues(f, sigma)
    comps = oracle.hessian3d(f, sigma)
    rng = np.random.default_rng(3)
    for _ in range(40):
        p = tuple(int(rng.integers(0, s)) for s in f.shape)
        zz, yy, xx, zy, zx, yx = (c[p] for c in comps)
        jac = _jacobi_eigvals([[zz, zy, zx], [zy, yy, yx], [zx, yx, xx]])
        got = np.array([e[p] for e in ev])
        assert np.allclose(got, jac, rtol=1e-10, atol=1e-12 * np.abs(jac).max())
    # ascending, and the trace is the Laplacian of Gaussian
    assert (ev[0] <= ev[1]).all() and (ev[1] <= ev[2]).all()
    log = oracle.filterbank3d(f, [(oracle.LOG, sigma)])[0]
    assert np.allclose(ev[0] + ev[1] + ev[2], log, rtol=1e-10, atol=1e-12 * np.abs(log).max())


def test_hessian_of_separable_quadratic_is_diagonal():
    """f = a z^2 + b y^2 + c x^2: every mixed derivative vanishes (the first
    derivative taps sum to zero), so the eigenvalues are the sorted diagonal."""
    n = 24
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    f = 0.5 * z * z - 1.5 * y * y + 0.25 * x * x
    sigma = 1.0
    zz, yy, xx, zy, zx, yx = oracle.hessian3d(f, sigma)
    inner = (slice(5, n - 5),) * 3
    for m in (zy, zx, yx):
        assert np.abs(m[inner]).max() < 1e-9
    ev = oracle.hessian_eigenvalues(f, sigma)
    diag = np.sort(np.stack([zz[inner], yy[inner], xx[inner]], -1), -1)
    for i in range(3):
        assert np.allclose(ev[i][inner], diag[..., i], rtol=1e-9, atol=1e-9)
    # closed form away from the faces, with the derivative taps not
    # re-normalised: per axis, g2 applied to u^2 gives S0 u^2 + S2 and to a
    # constant S0; g0 applied to u^2 gives u^2 + M (first moments vanish)
    k = np.arange(-3, 4, dtype=np.float64)
    g0 = np.exp(-0.5 * k * k)
    g0 /= g0.sum()
    g2 = (k * k - 1.0) * g0
    S0, S2, M = g2.sum(), (g2 * k * k).sum(), (g0 * k * k).sum()
    a, b, c = 0.5, -1.5, 0.25
    Z, Y, X = z[inner], y[inner], x[inner]
    assert np.allclose(zz[inner], a * (S0 * Z * Z + S2) + S0 * (b * (Y * Y + M) + c * (X * X + M)), rtol=1e-9)
    assert np.allclose(yy[inner], b * (S0 * Y * Y + S2) + S0 * (a * (Z * Z + M) + c * (X * X + M)), rtol=1e-9)
    assert np.allclose(xx[inner], c * (S0 * X * X + S2) + S0 * (a * (Z * Z + M) + b * (Y * Y + M)), rtol=1e-9)


# ------------------------------------------------------------ box statistics

def _brute_sums(f, w):
    p = np.pad(f.astype(np.float64), w, mode="symmetric")
    s1 = np.zeros(f.shape)
    s2 = np.zeros(f.shape)
    n0, n1, n2 = f.shape
    for dz in range(2 * w + 1):
        for dy in range(2 * w + 1):
            for dx in range(2 * w + 1):
                v = p[dz:dz + n0, dy:dy + n1, dx:dx + n2]
                s1 += v
                s2 += v * v
    return s1, s2


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("shape,w", [((6, 7, 8), 1), ((5, 9, 4), 2), ((3, 2, 5), 3)])
def test_box_sums_vs_brute_force(dtype, shape, w):
    f = _rand(shape, 4, dtype)
    s1, s2 = oracle.box_sums(f, w)
    b1, b2 = _brute_sums(f, w)
    if dtype in (np.uint8, np.uint16):
        assert np.array_equal(s1, b1) and np.array_equal(s2, b2)    # exact integers
    else:
        assert np.allclose(s1, b1, rtol=1e-12, atol=1e-12) and np.allclose(s2, b2, rtol=1e-12)


def test_box_mean_and_std_vs_scipy():
    f = _rand((7, 8, 9), 5)
    w = 1
    s1, s2 = oracle.box_sums(f, w)
    n = (2 * w + 1) ** 3
    assert np.allclose(s1 / n, nd.uniform_filter(f, 2 * w + 1, mode="reflect"), rtol=1e-12, atol=1e-12)
    std = nd.generic_filter(f, np.std, size=2 * w + 1, mode="reflect")
    m = s1 / n
    assert np.allclose(np.sqrt(np.maximum(s2 / n - m * m, 0)), std, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("method,k,c", [(oracle.LOCAL_MEAN, 0.0, 100.0), (oracle.LOCAL_NIBLACK, -0.2, 0.0),
                                        (oracle.LOCAL_NIBLACK, 0.5, 0.0), (oracle.LOCAL_SAUVOLA, 0.3, 32768.0)])
def test_threshold_box_vs_numpy_definition(method, k, c):
    f = _rand((8, 9, 10), 6, np.uint16)
    w = 2
    out, thr = oracle.threshold_box(f, method, w, k, c, return_threshold=True)
    p = np.pad(f.astype(np.float64), w, mode="symmetric")
    win = np.lib.stride_tricks.sliding_window_view(p, (2 * w + 1,) * 3)
    m = win.mean(axis=(-3, -2, -1))
    s = win.std(axis=(-3, -2, -1))
    if method == oracle.LOCAL_MEAN:
        t = m - c
    elif method == oracle.LOCAL_NIBLACK:
        t = m + k * s
    else:
        t = m * (1 + k * (s / c - 1))
    assert np.allclose(thr, t, rtol=1e-9, atol=1e-6)
    far = np.abs(f - t) > 1e-6 * (1 + np.abs(t))
    assert np.array_equal(out[far], (f > t)[far].astype(np.uint8))
    assert far.mean() > 0.99


def test_threshold_box_constant_volume_closed_forms():
    f = np.full((6, 7, 8), 1000, np.uint16)
    assert oracle.threshold_box(f, oracle.LOCAL_MEAN, 2, 0.0, 5.0).all()       # f > f - 5
    assert not oracle.threshold_box(f, oracle.LOCAL_MEAN, 2, 0.0, -5.0).any()  # f > f + 5
    assert not oracle.threshold_box(f, oracle.LOCAL_NIBLACK, 2, 0.7, 0.0).any()  # s = 0: f > f
    assert oracle.threshold_box(f, oracle.LOCAL_SAUVOLA, 2, 0.3, 128.0).all()  # T = 0.7 f
