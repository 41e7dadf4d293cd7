"""FP64 reference of the patch-denoising experiment of Sec. IV (TEST
INFRASTRUCTURE ONLY, see the package docstring).

Every stride-1 p x p patch of the noisy image is coded with error-driven
2D-OMP (stop once ||R||_F <= eps, at most s atoms; eps = 1.15 sigma p, the
paper's 1.15 sigma sqrt(m) with m = p^2 pixels), after removing its mean; the
image is rebuilt by averaging the overlapping reconstructions (mean added
back), and scored by PSNR and SSIM (Wang, Bovik, Sheikh, Simoncelli 2004, the
index Table III reports).
"""
from __future__ import annotations

import numpy as np

from .sdl_oracle import omp2d, reconstruct

__all__ = ["extract_patches", "patch_average", "psnr", "ssim", "gaussian_window", "denoise"]

SSIM_K1, SSIM_K2 = 0.01, 0.03      # stabilising constants of the SSIM index
SSIM_WIN, SSIM_SIGMA = 11, 1.5      # circular Gaussian window, normalised to sum 1


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


def gaussian_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA):
    """size x size Gaussian weights exp(-(u^2 + v^2) / (2 sigma^2)) about the
    centre, normalised to sum 1."""
    u = np.arange(size) - (size - 1) / 2.0
    w = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2.0 * sigma * sigma))
    return w / w.sum()


def ssim(x, ref, peak: float = 255.0) -> float:
    """Mean SSIM over every window position fully inside the image (valid
    region): per window, with Gaussian-weighted means mu, variances and
    covariance (weights w, sum 1),
      ((2 mu_x mu_y + C1)(2 cov + C2)) / ((mu_x^2 + mu_y^2 + C1)(var_x + var_y + C2)),
    C1 = (K1 peak)^2, C2 = (K2 peak)^2."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(ref, dtype=np.float64)
    w = gaussian_window()
    g = w.shape[0]
    H, W = x.shape
    C1, C2 = (SSIM_K1 * peak) ** 2, (SSIM_K2 * peak) ** 2
    total = 0.0
    for r in range(H - g + 1):
        for c in range(W - g + 1):
            a = x[r:r + g, c:c + g]
            b = y[r:r + g, c:c + g]
            mx, my = np.sum(w * a), np.sum(w * b)
            vx = np.sum(w * (a - mx) ** 2)
            vy = np.sum(w * (b - my) ** 2)
            cxy = np.sum(w * (a - mx) * (b - my))
            total += ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return float(total / ((H - g + 1) * (W - g + 1)))


def denoise(noisy, D1, D2, s: int, eps: float):
    """Code every patch with (D1, D2) and rebuild the image."""
    H, W = noisy.shape
    p = D1.shape[0]
    Y, means = extract_patches(noisy, p)
    code = omp2d(Y, D1, D2, s, eps=eps)
    rec = reconstruct(D1, D2, code.support, code.coef) + means[:, None, None]
    return patch_average(rec, H, W), code
