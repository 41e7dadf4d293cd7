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


@pytest.mark.parametrize("M,N,K,ldc", [(300, 200, 192, 204), (1000, 512, 256, 512), (77, 13, 8, 13),
                                       (77, 13, 8, 16), (64, 20, 8, 20), (4096, 576, 512, 576)])
def test_gemm_tensor_map_outputs(gpu_ctx, M, N, K, ldc):
    """FP32 and BF16 outputs alone (the tensor-map stores, a reduce-add when
    accumulating; rows that are not whole 16-byte units, N = 13 and the BF16
    output at N = 20, take the transpose path): every element of the M x N
    block right, the padding of each row untouched."""
    A, An = bf16_pair((M, K), 6)
    B, Bn = bf16_pair((N, K), 7)
    bias = torch.randn(N, generator=torch.Generator().manual_seed(8))
    alpha = -1.25
    Cfull = torch.full((M, ldc), 2.0, device="cuda:0")
    C = Cfull[:, :N]
    sdl.gemm_bf16(gpu_ctx, A, B, alpha=alpha, bias=bias.cuda(), act=1, C=C, accumulate=True)
    Cbfull = torch.full((M, ldc + 8 - ldc % 8 if ldc % 8 else ldc), 7.0, dtype=torch.bfloat16,
                        device="cuda:0")
    Cb = Cbfull[:, :N]
    sdl.gemm_bf16(gpu_ctx, A, B, alpha=alpha, bias=bias.cuda(), act=1, Cb=Cb)
    C2 = sdl.gemm_bf16(gpu_ctx, A, B, alpha=alpha)
    assert gpu_ctx.status() == 0
    z = alpha * (An @ Bn.T) + bias.double().numpy()[None, :]
    erf = np.vectorize(math.erf)
    g = 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))
    assert np.abs(C.cpu().numpy() - (g + 2.0)).max() < 1e-4 * (np.abs(g).max() + 2.0)
    assert np.abs(Cb.float().cpu().numpy() - g).max() < 1e-2 * np.abs(g).max()
    assert np.abs(C2.cpu().numpy() - alpha * (An @ Bn.T)).max() < 2e-5 * np.abs(z).max()
    assert bool((Cfull[:, N:] == 2.0).all())
    assert bool((Cbfull[:, N:].float() == 7.0).all())


def test_gemm_ragged_k_ignores_row_padding(gpu_ctx):
    """K = 13 inside rows of 16: the operand loads stop at column K, so huge
    values in the padding columns change nothing."""
    M, N, K, ld = 200, 136, 13, 16
    g = torch.Generator().manual_seed(9)
    A = torch.full((M, ld), 1e30).to(torch.bfloat16)
    B = torch.full((N, ld), 1e30).to(torch.bfloat16)
    A[:, :K] = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B[:, :K] = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = sdl.gemm_bf16(gpu_ctx, A.cuda()[:, :K], B.cuda()[:, :K])
    assert gpu_ctx.status() == 0
    ref = A[:, :K].double().numpy() @ B[:, :K].double().numpy().T
    assert np.abs(C.cpu().numpy() - ref).max() < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("M,N,K,terms", [(1000, 4096, 1024, 3), (300, 200, 192, 2), (77, 13, 8, 3),
                                         (256, 384, 512, 1)])
def test_gemm_terms_sum_in_one_accumulator(gpu_ctx, M, N, K, terms):
    """sdl_gemm_bf16_terms: the sum of 1 to 3 products in one accumulator
    (plain FP32 output, an accumulating one with bias and GELU, and the BF16
    copy) against the FP64 sum of the same BF16-rounded operands."""
    ops = [(bf16_pair((M, K), 20 + t), bf16_pair((N, K), 40 + t)) for t in range(terms)]
    A = [a for (a, _), _ in ops]
    B = [b for _, (b, _) in ops]
    ref = sum(an @ bn.T for (_, an), (_, bn) in ops)
    C = sdl.gemm_bf16_terms(gpu_ctx, A, B)
    bias = torch.randn(N, generator=torch.Generator().manual_seed(11))
    C2 = torch.full((M, N), -1.5, device="cuda:0")
    Cb = torch.empty((M, N + (-N) % 8), dtype=torch.bfloat16, device="cuda:0")[:, :N]
    sdl.gemm_bf16_terms(gpu_ctx, A, B, alpha=0.5, bias=bias.cuda(), act=1, C=C2,
                        accumulate=True, Cb=Cb)
    assert gpu_ctx.status() == 0
    scale = np.abs(ref).max()
    assert np.abs(C.cpu().numpy() - ref).max() < 2e-5 * scale
    z = 0.5 * ref + bias.double().numpy()[None, :]
    g = 0.5 * z * (1.0 + torch.special.erf(torch.from_numpy(z / math.sqrt(2.0))).numpy())
    assert np.abs(C2.cpu().numpy() - (g - 1.5)).max() < 1e-4 * (np.abs(g).max() + 1.5)
    assert np.abs(Cb.float().cpu().numpy() - g).max() < 1e-2 * np.abs(g).max()


def test_gemm_terms_rejects_bad_counts(gpu_ctx):
    """Four operand pairs, or lists of unequal length, are argument errors
    checked on the host before any launch."""
    A = [torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda:0") for _ in range(4)]
    with pytest.raises(sdl.SDLError):
        sdl.gemm_bf16_terms(gpu_ctx, A, A)
    with pytest.raises(ValueError):
        sdl.gemm_bf16_terms(gpu_ctx, A[:2], A[:1])
    assert gpu_ctx.status() == 0
