"""Pins of the oracle's denoising pipeline (Sec. IV) against brute force and
closed forms."""
import numpy as np

import oracle
from oracle import denoise as dn
from paper_2007_03800_gb300 import synth


def test_patches_are_windows_minus_mean():
    img = np.arange(7 * 9, dtype=float).reshape(7, 9) ** 1.5
    Y, means = dn.extract_patches(img, 3)
    assert Y.shape == (5 * 7, 3, 3)
    k = 2 * 7 + 4                                   # corner (2, 4)
    win = img[2:5, 4:7]
    assert np.allclose(Y[k], win - win.mean()) and np.isclose(means[k], win.mean())
    assert np.allclose(Y.mean(axis=(1, 2)), 0.0, atol=1e-12)


def test_average_of_exact_patches_is_the_image():
    img = synth.synthetic_image(3, size=40)
    Y, means = dn.extract_patches(img, 6)
    back = dn.patch_average(Y + means[:, None, None], 40, 40)
    assert np.allclose(back, img, atol=1e-12)


def test_average_weights_by_brute_force():
    """Replace patch k by the constant k: each pixel is the mean index of the
    patches that cover it, computed here pixel by pixel."""
    H, W, p = 9, 11, 4
    N = (H - p + 1) * (W - p + 1)
    pat = np.arange(N, dtype=float)[:, None, None] * np.ones((1, p, p))
    out = dn.patch_average(pat, H, W)
    for y in range(H):
        for x in range(W):
            ks = [r * (W - p + 1) + c for r in range(H - p + 1) for c in range(W - p + 1)
                  if r <= y < r + p and c <= x < c + p]
            assert np.isclose(out[y, x], np.mean(ks))


def test_psnr_closed_form():
    ref = np.full((8, 8), 100.0)
    assert np.isclose(dn.psnr(ref + 1.0, ref), 20 * np.log10(255.0))
    assert np.isclose(dn.psnr(ref + 2.0, ref, peak=1.0), 10 * np.log10(1 / 4.0))


def test_denoise_with_orthonormal_dictionary_is_thresholding():
    """Orthonormal D1 = D2 = I: error-driven OMP keeps the largest pixels of
    each mean-removed patch until the residual drops below eps (Remark 1's
    T_s with a data-driven s); with eps = 0 and s = p^2 the image comes back."""
    img = synth.synthetic_image(5, size=24)
    I = np.eye(4)
    back, code = dn.denoise(img, I, I, 16, eps=1e-9)
    assert np.allclose(back, img, atol=1e-9)
    Y, _ = dn.extract_patches(img, 4)
    r = oracle.residual(Y, I, I, code.support, code.coef)
    assert np.all(np.sqrt(np.sum(r * r, axis=(1, 2))) <= 1e-9 + 1e-12)


def test_ssim_identity_and_symmetry():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 255, (20, 23))
    y = np.clip(x + rng.normal(0, 15, x.shape), 0, 255)
    assert np.isclose(dn.ssim(x, x), 1.0, atol=1e-12)
    assert np.isclose(dn.ssim(x, y), dn.ssim(y, x), rtol=1e-12)
    assert dn.ssim(x, y) < 1.0


def test_ssim_of_constant_images_closed_form():
    """Constant images a and b: every window has zero variances, so SSIM is the
    luminance term (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 100.0, 140.0
    C1 = (0.01 * 255) ** 2
    got = dn.ssim(np.full((15, 15), a), np.full((15, 15), b))
    assert np.isclose(got, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_ssim_by_brute_force_weighted_sums():
    """One window position (11 x 11 image), the weights written out from the
    Gaussian formula and every moment summed term by term."""
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 255, (11, 11))
    y = rng.uniform(0, 255, (11, 11))
    w = np.array([[np.exp(-((i - 5) ** 2 + (j - 5) ** 2) / 4.5) for j in range(11)] for i in range(11)])
    w /= w.sum()
    mx = sum(w[i, j] * x[i, j] for i in range(11) for j in range(11))
    my = sum(w[i, j] * y[i, j] for i in range(11) for j in range(11))
    vx = sum(w[i, j] * x[i, j] ** 2 for i in range(11) for j in range(11)) - mx * mx
    vy = sum(w[i, j] * y[i, j] ** 2 for i in range(11) for j in range(11)) - my * my
    cxy = sum(w[i, j] * x[i, j] * y[i, j] for i in range(11) for j in range(11)) - mx * my
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    want = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    assert np.isclose(dn.ssim(x, y), want, rtol=1e-10)
