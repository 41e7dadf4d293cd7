"""Precision extension: BF16 tensor-core correlations with FP32 re-scoring,
and FP64 normal-equation solves, each result against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_03800_gb300 import sdl, synth
from parity import (COEF_RTOL, DICT_RTOL, RMSE_RTOL, codes_from_oracle, coef_rel_error,
                    compare_supports, to_gpu_problem)

pytestmark = pytest.mark.gpu


@pytest.fixture
def prec_ctx():
    ctx = sdl.Context(0)
    yield ctx
    ctx.close()


def hsi_problem(N, seed=31):
    Y = synth.hyperspectral(N, seed=seed)            # 16 x 64 signals
    D1, D2 = synth.init_dictionaries(16, 64, 32, 128, seed=1)
    return Y, D1, D2


def test_bf16_correlation_error_within_bound(prec_ctx):
    """The tensor-core C0 obeys the stated bound |dC0| <= 2^-7 (1.03) ||Y||_F."""
    Y, D1, D2 = hsi_problem(300)
    ref = np.einsum("ai,kab,bj->kij", D1, Y, D2)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    C0 = torch.empty((300, 32 * 128), dtype=torch.float32, device="cuda:0")
    # C0 through the public GEMM with the same operands the coder uses
    Yb = Yg.transpose(1, 2).reshape(300, -1).contiguous().to(torch.bfloat16)
    KT = torch.einsum("ai,bj->jiba", torch.tensor(D1), torch.tensor(D2)).reshape(32 * 128, -1)
    KT = KT.to(torch.float32).to(torch.bfloat16).contiguous().cuda()
    sdl.gemm_bf16(prec_ctx, Yb, KT, C=C0)
    got = C0.cpu().numpy().reshape(300, 128, 32).transpose(0, 2, 1)
    bound = 2.0 ** -7 * 1.03 * np.linalg.norm(Y, axis=(1, 2))
    assert np.all(np.abs(got - ref) <= bound[:, None, None])


def test_bf16_rescored_picks_match_oracle(prec_ctx):
    Y, D1, D2 = hsi_problem(257)
    ref = oracle.omp2d(Y, D1, D2, 10)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    prec_ctx.set_precision(sdl.Context.PREC_BF16_CORR)
    out = prec_ctx.sparse_code(Yg, D1g, D2g, 10)
    assert prec_ctx.status() == 0
    assert prec_ctx.precision_stats() > 0
    rep, exact = compare_supports(out.support.cpu().numpy(), out.nnz.cpu().numpy(), ref)
    assert rep.bad == 0 and rep.ties <= 2, rep
    assert coef_rel_error(out.coef.cpu().numpy(), ref.coef, exact).max() < COEF_RTOL
    # without re-scoring, BF16 picks drift from the FP32/FP64 picks
    prec_ctx.set_precision(sdl.Context.PREC_BF16_CORR | sdl.Context.PREC_NO_RESCORE)
    raw = prec_ctx.sparse_code(Yg, D1g, D2g, 10)
    rep_raw, _ = compare_supports(raw.support.cpu().numpy(), raw.nnz.cpu().numpy(), ref)
    assert rep_raw.exact < rep.exact, (rep_raw, rep)


@pytest.mark.parametrize("side", [1, 2])
def test_fp64_solve_matches_oracle(prec_ctx, side):
    Y, D1, D2 = hsi_problem(600, seed=33)
    ref_code = oracle.omp2d(Y, D1, D2, 10)
    upd = (oracle.update_D1 if side == 1 else oracle.update_D2)(Y, D1, D2, ref_code.support,
                                                                ref_code.coef)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    codes = codes_from_oracle(ref_code.support, ref_code.coef)
    prec_ctx.set_precision(sdl.Context.PREC_FP64_SOLVE)
    obj = torch.zeros(2, dtype=torch.float32, device="cuda:0")
    (prec_ctx.update_D1 if side == 1 else prec_ctx.update_D2)(Yg, D1g, D2g, codes, objective_out=obj)
    assert prec_ctx.status() == 0
    D = (D1g if side == 1 else D2g).cpu().numpy()
    assert np.abs(D - upd.D).max() < DICT_RTOL
    assert abs(obj.cpu().numpy()[1] - upd.obj_after) / upd.obj_after < 1e-4


def test_bf16_fp64_iteration_matches_oracle(prec_ctx):
    Y, D1, D2 = hsi_problem(800, seed=35)
    ref = oracle.iterate(Y, D1, D2, 10)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    prec_ctx.set_precision(sdl.Context.PREC_BF16_CORR | sdl.Context.PREC_FP64_SOLVE)
    rmse = torch.zeros(2, dtype=torch.float32, device="cuda:0")
    out = prec_ctx.iterate(Yg, D1g, D2g, 10, rmse_out=rmse)
    assert prec_ctx.status() == 0
    r = rmse.cpu().numpy()
    assert abs(r[1] - ref.rmse_after_D2) / ref.rmse_after_D2 < RMSE_RTOL
    assert np.abs(D1g.cpu().numpy() - ref.D1).max() < DICT_RTOL
    assert np.abs(D2g.cpu().numpy() - ref.D2).max() < DICT_RTOL
