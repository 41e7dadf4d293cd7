"""FP64 reference of the patch-denoising experiment of Sec. IV (TEST
INFRASTRUCTURE ONLY, see the package docstring).

Every stride-1 p x p patch of the noisy image is coded with error-driven
2D-OMP (stop once ||R||_F <= eps, at most s atoms; eps = 1.15 sigma p, the
paper's 1.15 sigma sqrt(m) with m = p^2 pixels), after removing its mean; the
image is rebuilt by averaging the overlapping reconstructions (mean added
back), and scored by PSNR.
"""
from __future__ import annotations

import numpy as np

from .sdl_oracle import omp2d, reconstruct

__all__ = ["extract_patches", "patch_average", "psnr", "denoise"]


def extract_patches(img, p: int):
    """Patches in raster order of their top-left corner (r, c):
    Y[k] = img[r:r+p, c:c+p] - mean, k = r*(W-p+1) + c.  Returns (Y, means)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    Y = np.empty(((H - p + 1) * (W - p + 1), p, p))
    k = 0
    for r in range(H - p + 1):
        for c in range(W - p + 1):
            Y[k] = img[r:r + p, c:c + p]
            k += 1
    means = Y.mean(axis=(1, 2))
    return Y - means[:, None, None], means


def patch_average(patches, H: int, W: int):
    """Pixel = plain average of every (already mean-restored) patch covering it."""
    N, p, _ = patches.shape
    acc = np.zeros((H, W))
    cnt = np.zeros((H, W))
    k = 0
    for r in range(H - p + 1):
        for c in range(W - p + 1):
            acc[r:r + p, c:c + p] += patches[k]
            cnt[r:r + p, c:c + p] += 1
            k += 1
    return acc / cnt


def psnr(x, ref, peak: float = 255.0) -> float:
    mse = np.mean((np.asarray(x, dtype=np.float64) - np.asarray(ref, dtype=np.float64)) ** 2)
    return float(10.0 * np.log10(peak * peak / mse))


def denoise(noisy, D1, D2, s: int, eps: float):
    """Code every patch with (D1, D2) and rebuild the image."""
    H, W = noisy.shape
    p = D1.shape[0]
    Y, means = extract_patches(noisy, p)
    code = omp2d(Y, D1, D2, s, eps=eps)
    rec = reconstruct(D1, D2, code.support, code.coef) + means[:, None, None]
    return patch_average(rec, H, W), code
