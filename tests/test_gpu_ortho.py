"""Orthonormal variant (Remark 1) on the GPU against the FP64 oracle:
thresholded codes, one Algorithm-1 iteration with Procrustes updates, a
ten-iteration RMSE trajectory, and the rank-deficient case."""
import numpy as np
import pytest
import torch

import oracle
from oracle import ortho
from paper_2007_03800_gb300 import sdl
from parity import COEF_RTOL, DICT_RTOL, RMSE_RTOL, TIE_REL, to_gpu_problem

pytestmark = pytest.mark.gpu


def orth(seed, p):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((p, p)))
    return Q * np.sign(np.diag(R))


def ortho_model(N, p, s, snr_db=20.0, seed=61):
    """Y_k = Q1 X_k Q2^T + noise with orthonormal Q1, Q2 and s planted pairs."""
    rng = np.random.default_rng(seed)
    Q1, Q2 = orth(seed + 1, p), orth(seed + 2, p)
    keys = rng.random((N, p * p))
    sup = np.argsort(keys, axis=1)[:, :s].astype(np.int64)
    coef = rng.standard_normal((N, s))
    clean = oracle.reconstruct(Q1, Q2, sup, coef)
    e = np.einsum("kab,kab->k", clean, clean)
    sigma = np.sqrt(e / (p * p * 10 ** (snr_db / 10)))
    return clean + rng.standard_normal(clean.shape) * sigma[:, None, None]


def compare_threshold(gpu_sup, Y, D1, D2, ref_sup):
    """Pick-by-pick equality; at the first difference the two pairs must be
    tied in the oracle's |C| within TIE_REL.  Returns (exact mask, ties)."""
    C = np.abs(np.einsum("ai,kab,bj->kij", D1, Y, D2)).transpose(0, 2, 1).reshape(len(Y), -1)
    same = np.all(gpu_sup == ref_sup, axis=1)
    ties = 0
    for k in np.nonzero(~same)[0]:
        t = np.nonzero(gpu_sup[k] != ref_sup[k])[0][0]
        a, b = C[k, gpu_sup[k, t]], C[k, ref_sup[k, t]]
        assert abs(a - b) <= TIE_REL * max(a, b), (k, t, a, b)
        ties += 1
    return same, ties


@pytest.mark.parametrize("p,s", [(8, 4), (12, 6), (6, 3), (8, 20)])
def test_threshold_codes_match_oracle(gpu_ctx, p, s):
    """Compiled square shapes (8, 12 with s <= 16) and the generic kernel
    (6 x 6; s = 20 > 16)."""
    Y = ortho_model(4096, p, s)
    D1, D2 = orth(1, p), orth(2, p)
    sup, coef, res = ortho.threshold_code(Y, D1, D2, s)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    out = gpu_ctx.ortho_sparse_code(Yg, D1g, D2g, s)
    assert gpu_ctx.status() == 0
    same, ties = compare_threshold(out.support.cpu().numpy(), Y, D1, D2, sup)
    assert ties <= 4
    c = out.coef.cpu().numpy().astype(np.float64)[same]
    err = np.linalg.norm(c - coef[same], axis=1) / np.linalg.norm(coef[same], axis=1)
    assert err.max() < COEF_RTOL
    r = out.res_energy.cpu().numpy().astype(np.float64)[same]
    assert np.all(np.abs(r - res[same]) <= 1e-5 * np.einsum("kab,kab->k", Y, Y)[same])


@pytest.mark.parametrize("p,s", [(8, 4), (12, 6), (16, 8)])
def test_ortho_iteration_matches_oracle(gpu_ctx, p, s):
    Y = ortho_model(3000, p, s, seed=62 + p)
    D1, D2 = orth(1, p), orth(2, p)
    ref = ortho.ortho_iterate(Y, D1, D2, s)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    out = gpu_ctx.ortho_iterate(Yg, D1g, D2g, s, rmse_out=rmse)
    assert gpu_ctx.status() == 0
    r = rmse.cpu().numpy()
    assert abs(r[0] - ref.rmse_after_D1) / ref.rmse_after_D1 < RMSE_RTOL, (r, ref.rmse_after_D1)
    assert abs(r[1] - ref.rmse_after_D2) / ref.rmse_after_D2 < RMSE_RTOL, (r, ref.rmse_after_D2)
    G1, G2 = D1g.cpu().numpy(), D2g.cpu().numpy()
    assert np.abs(G1 - ref.D1).max() < DICT_RTOL
    assert np.abs(G2 - ref.D2).max() < DICT_RTOL
    assert np.allclose(G1.T @ G1, np.eye(p), atol=1e-5)
    same, ties = compare_threshold(out.support.cpu().numpy(), Y, ref.D1, D2, ref.support)
    assert ties <= 4


def test_ortho_ten_iterations_rmse_trajectory(gpu_ctx):
    p, s = 8, 4
    Y = ortho_model(4096, p, s, seed=70)
    D1, D2 = orth(1, p), orth(2, p)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    out = None
    for it in range(10):
        ref = ortho.ortho_iterate(Y, D1, D2, s)
        D1, D2 = ref.D1, ref.D2
        out = gpu_ctx.ortho_iterate(Yg, D1g, D2g, s, out=out, rmse_out=rmse)
        r = rmse.cpu().numpy()
        assert abs(r[1] - ref.rmse_after_D2) / ref.rmse_after_D2 < RMSE_RTOL, (it, r, ref.rmse_after_D2)
    assert gpu_ctx.status() == 0


def test_rank_deficient_procrustes_is_flagged_and_leaves_the_dictionary(gpu_ctx):
    """Signals orthogonal to atom p-1 of D1: no code uses it, column p-1 of B1
    is zero, the Procrustes problem has no unique solution."""
    p, s = 8, 3
    rng = np.random.default_rng(71)
    D1, D2 = orth(1, p), orth(2, p)
    Y = rng.standard_normal((2000, p, p))
    d = D1[:, p - 1]
    Y = Y - np.einsum("a,b,kbc->kac", d, d, Y)     # D1[:, p-1]^T Y_k = 0
    with pytest.raises(oracle.SingularError):
        sup, coef, _ = ortho.threshold_code(Y, D1, D2, s)
        ortho.procrustes_D1(Y, D1, D2, sup, coef)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    before = D1g.cpu().numpy().copy()
    gpu_ctx.ortho_iterate(Yg, D1g, D2g, s)
    assert sdl.ERRORS[gpu_ctx.status()] == "SDL_ERR_SINGULAR"
    assert np.array_equal(D1g.cpu().numpy(), before)
