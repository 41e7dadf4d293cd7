"""The tcgen05 BF16 GEMM (sdl_gemm_bf16) against an FP64 product of the same
BF16-rounded operands, with every epilogue option."""
import math

import numpy as np
import pytest
import torch

from paper_2007_03800_gb300 import sdl

pytestmark = pytest.mark.gpu


def bf16_pair(shape, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(shape, generator=g)
    xb = x.to(torch.bfloat16)
    return xb.cuda(), xb.float().double().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 512), (200, 300, 144),
                                   (4096, 576, 512), (77, 13, 8)])
def test_gemm_matches_fp64(gpu_ctx, M, N, K):
    A, An = bf16_pair((M, K), 1)
    B, Bn = bf16_pair((N, K), 2)
    C = sdl.gemm_bf16(gpu_ctx, A, B)
    assert gpu_ctx.status() == 0
    ref = An @ Bn.T
    err = np.abs(C.cpu().numpy() - ref).max() / (np.abs(ref).max() + 1e-30)
    assert err < 2e-5, err


def test_gemm_epilogues(gpu_ctx):
    M, N, K = 300, 200, 192
    A, An = bf16_pair((M, K), 3)
    B, Bn = bf16_pair((N, K), 4)
    bias = torch.randn(N, generator=torch.Generator().manual_seed(5))
    alpha = 0.37
    C = torch.full((M, N), 2.0, device="cuda:0")
    Cb = torch.empty((M, N), dtype=torch.bfloat16, device="cuda:0")
    Ct = torch.empty((N, M + 8), dtype=torch.bfloat16, device="cuda:0")   # padded rows
    pre = torch.empty((M, N), device="cuda:0")
    sdl.gemm_bf16(gpu_ctx, A, B, alpha=alpha, bias=bias.cuda(), act=1, C=C, accumulate=True,
                  Cb=Cb, Ct=Ct, pre=pre)
    assert gpu_ctx.status() == 0
    z = alpha * (An @ Bn.T) + bias.double().numpy()[None, :]
    erf = np.vectorize(math.erf)
    g = 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))
    assert np.abs(pre.cpu().numpy() - z).max() < 1e-4 * np.abs(z).max()
    assert np.abs(C.cpu().numpy() - (g + 2.0)).max() < 1e-4 * np.abs(g).max()
    assert np.abs(Cb.float().cpu().numpy() - g).max() < 1e-2 * np.abs(g).max()
    assert np.abs(Ct[:, :M].float().cpu().numpy() - g.T).max() < 1e-2 * np.abs(g).max()
