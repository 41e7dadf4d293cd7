"""Denoising pipeline (Sec. IV) on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import denoise as dn
from paper_2007_03800_gb300 import denoise, sdl, synth
from parity import to_gpu_problem

pytestmark = pytest.mark.gpu


def noisy_image(size, seed=7, sigma=20.0):
    clean = synth.synthetic_image(seed, size=size)
    noisy = clean + np.random.default_rng(seed + 1).normal(0, sigma, clean.shape)
    return clean, noisy


def test_extract_patches_matches_oracle(gpu_ctx):
    _, noisy = noisy_image(50)
    for p in (8, 12, 16):
        Y, means = sdl.extract_patches(torch.tensor(noisy, dtype=torch.float32, device="cuda:0"), p)
        Yr, mr = dn.extract_patches(noisy, p)
        assert np.abs(Y.cpu().numpy() - Yr).max() < 2e-3
        assert np.abs(means.cpu().numpy() - mr).max() < 2e-3


def test_patch_average_and_psnr_match_oracle(gpu_ctx):
    clean, noisy = noisy_image(48)
    p, n, s = 8, 16, 4
    D1, D2 = synth.init_dictionaries(p, p, n, n, seed=1)
    ref_img, ref_code = dn.denoise(noisy, D1, D2, s, eps=1.15 * 20.0 * p)
    Yr, means = dn.extract_patches(noisy, p)
    _, D1g, D2g = to_gpu_problem(Yr[:1], D1, D2)
    codes = sdl.Codes(torch.tensor(ref_code.support, dtype=torch.int32, device="cuda:0"),
                      torch.tensor(ref_code.coef, dtype=torch.float32, device="cuda:0"),
                      torch.tensor(ref_code.nnz, dtype=torch.int32, device="cuda:0"))
    img = sdl.patch_average(gpu_ctx, codes, torch.tensor(means, dtype=torch.float32, device="cuda:0"),
                            D1g, D2g, p, 48, 48)
    assert np.abs(img.cpu().numpy() - ref_img).max() < 1e-3
    cl = torch.tensor(clean, dtype=torch.float32, device="cuda:0")
    got = sdl.psnr(img, cl).item()
    assert abs(got - dn.psnr(ref_img, clean)) < 1e-3


def test_pipeline_matches_oracle_small(gpu_ctx):
    """Three patch sizes learned together for 2 iterations on a 72x72 image:
    each group's dictionaries and PSNR follow the oracle run of the same
    steps (error-driven coding, Algorithm 1, averaging)."""
    clean, noisy = noisy_image(72, seed=11)
    sigma = 20.0
    res = denoise.denoise(gpu_ctx, torch.tensor(noisy, dtype=torch.float32, device="cuda:0"), sigma,
                          iterations=2, clean=torch.tensor(clean, dtype=torch.float32, device="cuda:0"))
    assert gpu_ctx.status() == 0
    for g, (p, n, s) in enumerate(denoise.DEFAULT_GROUPS):
        Y, _ = dn.extract_patches(noisy, p)
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=1)
        eps = 1.15 * sigma * p
        for _ in range(2):
            it = oracle.iterate(Y, D1, D2, s, eps=eps)
            D1, D2 = it.D1, it.D2
        ref_img, _ = dn.denoise(noisy, D1, D2, s, eps)
        ref_psnr = dn.psnr(ref_img, clean)
        assert abs(res["psnr"][g].item() - ref_psnr) < 0.02, (p, res["psnr"][g].item(), ref_psnr)
        assert np.abs(res["dictionaries"][g][0].cpu().numpy() - D1).max() < 2e-3


def test_pipeline_full_size_properties(gpu_ctx):
    """The mixed-batch denoising workload at full size: a 512x512 image with
    sigma = 20, all 255025 / 251001 / 247009 patches of 8x8 / 12x12 / 16x16,
    10 iterations.  Denoising must beat the noisy input by a clear margin,
    codes respect the cap, and the run reports no device error."""
    clean, noisy = noisy_image(512, seed=3)
    cl = torch.tensor(clean, dtype=torch.float32, device="cuda:0")
    nz = torch.tensor(noisy, dtype=torch.float32, device="cuda:0")
    res = denoise.denoise(gpu_ctx, nz, 20.0, iterations=10, clean=cl)
    assert gpu_ctx.status() == 0
    base = sdl.psnr(nz, cl).item()
    for g, (p, n, s) in enumerate(denoise.DEFAULT_GROUPS):
        assert res["psnr"][g].item() > base + 3.0, (p, res["psnr"][g].item(), base)
        assert 0.0 < res["nnz_mean"][g].item() <= s
        r = res["rmse"].cpu().numpy()
        assert np.all(np.isfinite(r))


def test_ssim_matches_oracle(gpu_ctx):
    rng = np.random.default_rng(12)
    clean = synth.synthetic_image(9, size=64)
    noisy = np.clip(clean + rng.normal(0, 20, clean.shape), 0, 255)
    want = dn.ssim(noisy, clean)
    cg = torch.tensor(clean, dtype=torch.float32, device="cuda:0")
    ng = torch.tensor(noisy, dtype=torch.float32, device="cuda:0")
    got = sdl.ssim(gpu_ctx, ng, cg).item()
    assert abs(got - want) < 1e-5, (got, want)
    assert abs(sdl.ssim(gpu_ctx, cg, cg).item() - 1.0) < 1e-6


@pytest.mark.parametrize("variant", ["general", "ortho"])
def test_table3_pipeline_matches_oracle(gpu_ctx, variant):
    """Fixed dictionaries (no learning), error-driven coding of every patch,
    averaging, PSNR and SSIM: the GPU pipeline against the oracle's."""
    from oracle import ortho as ortho_oracle
    from paper_2007_03800_gb300 import denoise as dn_gpu
    sigma, p, n = 20.0, 8, 16
    clean = synth.synthetic_image(10, size=48)
    noisy = clean + np.random.default_rng(13).normal(0, sigma, clean.shape)
    if variant == "general":
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=1)
    else:
        D1, D2 = dn_gpu.orthonormal_start(p, 1), dn_gpu.orthonormal_start(p, 2)
    eps = 1.15 * sigma * p
    Y, means = dn.extract_patches(noisy, p)
    if variant == "general":
        ref = oracle.omp2d(Y, D1, D2, p // 2, eps=eps)
        sup, coef = ref.support, ref.coef
    else:
        sup, coef, _ = ortho_oracle.threshold_code(Y, D1, D2, p // 2, eps=eps)
    rec = oracle.reconstruct(D1, D2, sup, coef) + means[:, None, None]
    want = dn.patch_average(rec, 48, 48)
    ng = torch.tensor(noisy, dtype=torch.float32, device="cuda:0")
    cg = torch.tensor(clean, dtype=torch.float32, device="cuda:0")
    Yg, mg = sdl.extract_patches(ng, p)
    D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device="cuda:0"))
    D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device="cuda:0"))
    if variant == "general":
        code = gpu_ctx.sparse_code(Yg, D1g, D2g, p // 2, eps=eps)
    else:
        code = gpu_ctx.ortho_sparse_code(Yg, D1g, D2g, p // 2, eps=eps)
    img = sdl.patch_average(gpu_ctx, code, mg, D1g, D2g, p, 48, 48)
    gpu_ctx.check()
    got = img.cpu().numpy().astype(np.float64)
    close = np.abs(got - want) < 1e-3
    assert close.mean() > 0.999, close.mean()
    assert abs(sdl.psnr(img, cg).item() - dn.psnr(want, clean)) < 1e-3
    assert abs(sdl.ssim(gpu_ctx, img, cg).item() - dn.ssim(want, clean)) < 1e-4
