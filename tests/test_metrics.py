"""The benchmark's SSIM (Sec. 4.1 reports PSNR and SSIM) against a direct transcription of
its definition (Wang et al. 2004) with scipy's Gaussian filter, and its closed-form cases."""
import numpy as np
import pytest
import torch

scipy_nd = pytest.importorskip("scipy.ndimage")
import bench  # noqa: E402


def ssim_reference(a, b):
    a = a.astype(np.float64) / 255.0
    b = b.astype(np.float64) / 255.0
    vals = []
    for c in range(a.shape[2]):
        x, y = a[..., c], b[..., c]
        f = lambda z: scipy_nd.gaussian_filter(z, 1.5, truncate=5 / 1.5, mode="constant")[5:-5, 5:-5]  # noqa: E731
        mx, my = f(x), f(y)
        sxx, syy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
        c1, c2 = 0.01 ** 2, 0.03 ** 2
        vals.append((((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))).mean())
    return float(np.mean(vals))


def test_ssim_matches_definition_and_closed_forms():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 256, (40, 36, 3), dtype=np.uint8)
    b = np.clip(a.astype(int) + rng.integers(-20, 21, a.shape), 0, 255).astype(np.uint8)
    got = bench.ssim_gpu(torch, torch.from_numpy(a), torch.from_numpy(b))
    assert abs(got - ssim_reference(a, b)) < 1e-9
    assert abs(bench.ssim_gpu(torch, torch.from_numpy(a), torch.from_numpy(a)) - 1.0) < 1e-12
    c = np.full((20, 20, 1), 100, np.uint8)
    d = np.full((20, 20, 1), 140, np.uint8)
    mx, my, c1 = 100 / 255, 140 / 255, 0.01 ** 2                # constant images: luminance term only
    want = (2 * mx * my + c1) / (mx * mx + my * my + c1)
    assert abs(bench.ssim_gpu(torch, torch.from_numpy(c), torch.from_numpy(d)) - want) < 1e-12
