"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rand_volume(dtype, shape, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.uint8:
        return rng.integers(0, 256, shape).astype(np.uint8)
    if dtype == np.uint16:
        return rng.integers(0, 65536, shape).astype(np.uint16)
    return (rng.standard_normal(shape) * 3).astype(dtype)


def f16_half_ulp(ref: np.ndarray) -> np.ndarray:
    """Half a float16 ulp at |ref| (the rounding bound of one f16 store)."""
    a = np.abs(ref).astype(np.float16).astype(np.float64)
    up = np.nextafter(a.astype(np.float16), np.float16(np.inf)).astype(np.float64)
    return 0.5 * (up - a)


def assert_filter_close(got: np.ndarray, ref: np.ndarray, what: str = ""):
    """FP32 filters: max |err| <= 1e-4 x (max - min of the FP64 result);
    f16 outputs additionally get half an f16 ulp of the reference."""
    rng = float(ref.max() - ref.min()) if ref.size else 0.0
    tol = 1e-4 * rng + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    if got.dtype == np.float16:
        bound = tol + f16_half_ulp(ref)
        bad = err > bound
    else:
        bad = err > tol
    assert not bad.any(), (f"{what}: max err {err.max():.3e} vs tol {tol:.3e} "
                           f"(range {rng:.3e}) at {np.argwhere(bad)[:3].tolist()}")
    return float(err.max()), rng
