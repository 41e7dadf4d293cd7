"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs come from the seeded generators only; expected values come from the
oracle only.  Supports must match pick for pick except at argmax ties and
stop thresholds the oracle itself shows (counted, bounded, and every step of
such a signal checked by the oracle's replay of its picks); coefficients,
residual energies, dictionaries and RMSE must match within 1e-4 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_03800_gb300 import sdl, synth
from parity import (COEF_RTOL, DICT_RTOL, RMSE_RTOL, check_codes, check_iteration,
                    codes_from_oracle, coef_rel_error, to_gpu_problem)

pytestmark = pytest.mark.gpu


def run_code(ctx, Y, D1, D2, s, eps=0.0):
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    out = ctx.sparse_code(Yg, D1g, D2g, s, eps=eps)
    assert ctx.status() == 0
    return (out.support.cpu().numpy(), out.coef.cpu().numpy(), out.nnz.cpu().numpy(),
            out.res_energy.cpu().numpy())


def check_code(ctx, Y, D1, D2, s, eps=None, ref=None):
    sup, coef, nnz, energy = run_code(ctx, Y, D1, D2, s, eps=eps or 0.0)
    rep = check_codes(Y, D1, D2, s, sup, nnz, coef, energy, eps=eps, ref=ref)
    rep.assert_ok()
    return rep


def iterate_and_check(ctx, Y, D1, D2, s, eps=None, ref=None, out=None, Ygpu=None):
    """One sdl_iterate on copies of (D1, D2), judged by check_iteration."""
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2) if Ygpu is None else Ygpu
    D1i, D2i = sdl.dictionary(D1g.clone()), sdl.dictionary(D2g.clone())
    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    got = ctx.iterate(Yg, D1i, D2i, s, eps=eps or 0.0, out=out, rmse_out=rmse)
    assert ctx.status() == 0
    return check_iteration(Y, D1, D2, s, got.support.cpu().numpy(), got.nnz.cpu().numpy(),
                           got.coef.cpu().numpy(), D1i.cpu().numpy(), D2i.cpu().numpy(),
                           rmse.cpu().numpy(), eps=eps, ref=ref)


# ----------------------------------------------------------------- sparse coding
@pytest.mark.parametrize("p1,p2,n1,n2,s,N", [
    (8, 8, 16, 16, 4, 4096),      # 8x8 Kronecker workload, 256 atom pairs
    (12, 12, 24, 24, 6, 3001),    # 12x12 patches, ragged count
    (16, 16, 32, 32, 8, 1003),
    (16, 64, 32, 128, 10, 257),   # hyperspectral shape: compiled sizes, 768-thread CTAs
    (8, 40, 16, 72, 6, 1111),     # the same tiling with run-time sizes, ragged 16 x 72 and count
    (6, 10, 12, 20, 5, 999),      # p1 != p2, n1 != n2
    (8, 8, 6, 6, 3, 500),         # undercomplete
    (8, 8, 16, 16, 1, 777),       # s = 1
    (4, 4, 8, 8, 8, 640),         # s = p1 p2 / 2
    (20, 20, 50, 50, 6, 300),     # 64 x 64 tile
    (40, 8, 100, 16, 4, 300),     # 128 x 32 tile
])
def test_sparse_code_matches_oracle(gpu_ctx, p1, p2, n1, n2, s, N):
    rng = np.random.default_rng(1000 + p1 * 7 + n2)
    Y = rng.standard_normal((N, p1, p2))
    D1, D2 = synth.init_dictionaries(p1, p2, n1, n2, seed=1)
    check_code(gpu_ctx, Y, D1, D2, s)


def test_sparse_code_kronecker_model_recovery(gpu_ctx):
    """Noisy planted codes (20 dB): GPU and oracle agree on every pick, so the
    recovery rate of the planted supports is identical."""
    Y, D1t, D2t, sup_true, _ = synth.kron_model(4096, 8, 8, 16, 16, 4, 20.0, seed=11)
    rep = check_code(gpu_ctx, Y, D1t, D2t, 4)
    ref = oracle.omp2d(Y, D1t, D2t, 4)
    sup, _, _, _ = run_code(gpu_ctx, Y, D1t, D2t, 4)
    rec_ref = np.mean([set(ref.support[k]) == set(sup_true[k]) for k in range(4096)])
    rec_gpu = np.mean([set(sup[k]) == set(sup_true[k]) for k in range(4096)])
    assert abs(rec_ref - rec_gpu) <= rep.ties / 4096


def test_sparse_code_noiseless_orthonormal_exact(gpu_ctx):
    rng = np.random.default_rng(5)
    p = 8
    Q1, _ = np.linalg.qr(rng.standard_normal((p, p)))
    Q2, _ = np.linalg.qr(rng.standard_normal((p, p)))
    N, s = 1000, 6
    sup = np.stack([rng.choice(p * p, s, replace=False) for _ in range(N)])
    coef = np.sign(rng.standard_normal((N, s))) * (0.5 + rng.random((N, s)))
    Y = oracle.reconstruct(Q1, Q2, sup, coef)
    gs, gc, gn, _ = run_code(gpu_ctx, Y, Q1, Q2, s)
    assert np.all(gn == s)
    for k in range(N):
        m = dict(zip(sup[k], coef[k]))
        assert set(gs[k]) == set(sup[k])
        assert np.allclose([m[q] for q in gs[k]], gc[k], rtol=1e-5, atol=1e-5)


def test_error_driven_mode(gpu_ctx):
    """Denoising-style error-bounded coding (Sec. IV): stop at ||R|| <= eps."""
    img = synth.synthetic_image(7, size=128)
    noisy = img + np.random.default_rng(8).normal(0, 20.0, img.shape)
    Y, _ = synth.all_patches(noisy, 8)
    Y = Y[::5][:3000]
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    eps = 1.15 * 20.0 * 8
    rep = check_code(gpu_ctx, Y, D1, D2, 4, eps=eps)
    assert rep.exact >= 0.99 * rep.n


# ------------------------------------------------------------ dictionary updates
@pytest.mark.parametrize("p1,p2,n1,n2,s,N", [
    (8, 8, 16, 16, 4, 4096),
    (12, 12, 24, 24, 6, 2000),
    (16, 64, 32, 128, 10, 600),
    (6, 10, 12, 20, 5, 999),
    (8, 16, 20, 48, 5, 700),     # n2 > 32: the large solve, one output per thread
    (8, 40, 16, 72, 6, 800),     # the large solve's 4 x 4 blocks over a ragged 40 x 72
])
@pytest.mark.parametrize("side", [1, 2])
def test_update_matches_oracle(gpu_ctx, p1, p2, n1, n2, s, N, side):
    Y, _, _, _, _ = synth.kron_model(N, p1, p2, n1, n2, s, 20.0, seed=21 + side)
    D1, D2 = synth.init_dictionaries(p1, p2, n1, n2, seed=1)
    ref_code = oracle.omp2d(Y, D1, D2, s)
    upd = (oracle.update_D1 if side == 1 else oracle.update_D2)(Y, D1, D2, ref_code.support,
                                                                ref_code.coef)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    codes = codes_from_oracle(ref_code.support, ref_code.coef)
    obj = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    (gpu_ctx.update_D1 if side == 1 else gpu_ctx.update_D2)(Yg, D1g, D2g, codes, objective_out=obj)
    assert gpu_ctx.status() == 0
    D = (D1g if side == 1 else D2g).cpu().numpy()
    assert np.abs(D - upd.D).max() < DICT_RTOL
    err = coef_rel_error(codes.coef.cpu().numpy(), upd.coef, np.ones(N, bool))
    assert err.max() < COEF_RTOL
    o = obj.cpu().numpy()
    assert abs(o[0] - upd.obj_before) / upd.obj_before < 1e-4
    assert abs(o[1] - upd.obj_after) / upd.obj_after < 1e-4
    # the untouched dictionary really is untouched
    other = (D2g if side == 1 else D1g).cpu().numpy()
    assert np.array_equal(other, np.asarray(D2 if side == 1 else D1, dtype=np.float32))


def test_update_keeps_unused_atom(gpu_ctx):
    Y, _, _, _, _ = synth.kron_model(1500, 8, 8, 16, 16, 4, 20.0, seed=31)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    ref_code = oracle.omp2d(Y, D1, D2, 4)
    sup, coef = ref_code.support.copy(), ref_code.coef.copy()
    coef[sup % 16 == 5] = 0.0                     # atom i = 5 of D1 carries no weight
    upd = oracle.update_D1(Y, D1, D2, sup, coef)
    assert not upd.used[5]
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    codes = codes_from_oracle(sup, coef)
    gpu_ctx.update_D1(Yg, D1g, D2g, codes)
    assert gpu_ctx.status() == 0
    got = D1g.cpu().numpy()
    assert np.array_equal(got[:, 5], np.asarray(D1[:, 5], dtype=np.float32))
    assert np.abs(got - upd.D).max() < DICT_RTOL


# ------------------------------------------------------------------ Algorithm 1
def test_iterate_one_step(gpu_ctx):
    Y, _, _, _, _ = synth.kron_model(4096, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    iterate_and_check(gpu_ctx, Y, D1, D2, 4)


def test_iterate_ten_steps_rmse_trajectory(gpu_ctx):
    """10 iterations on the 8x8 Kronecker workload: the RMSE after every
    dictionary update follows the oracle's within 1e-4 relative."""
    Y, _, _, _, _ = synth.kron_model(4096, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    out = None
    for it in range(10):
        ref = oracle.iterate(Y, D1, D2, 4)
        D1, D2 = ref.D1, ref.D2
        out = gpu_ctx.iterate(Yg, D1g, D2g, 4, out=out, rmse_out=rmse)
        r = rmse.cpu().numpy()
        assert abs(r[0] - ref.rmse_after_D1) / ref.rmse_after_D1 < RMSE_RTOL, (it, r, ref.rmse_after_D1)
        assert abs(r[1] - ref.rmse_after_D2) / ref.rmse_after_D2 < RMSE_RTOL, (it, r, ref.rmse_after_D2)
    assert gpu_ctx.status() == 0


def test_iterate_full_size_properties(gpu_ctx):
    """200k mean-removed 12x12 image patches, 12x24 dictionaries, s = 6 (the
    benchmark workload, same launch configuration): sampled signals match the
    oracle, and the closed-form RMSE equals the explicit residual of the
    returned (D1, D2, X)."""
    imgs = np.stack([synth.synthetic_image(100 + i) for i in range(8)])
    Y = synth.random_patches(imgs, 200_000, 12, seed=5)
    D1, D2 = synth.init_dictionaries(12, 12, 24, 24, seed=1)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    codes = gpu_ctx.sparse_code(Yg, D1g, D2g, 6)
    rows = np.random.default_rng(0).choice(200_000, 1500, replace=False)
    rep = check_codes(Y[rows], D1, D2, 6, codes.support.cpu().numpy()[rows], codes.nnz.cpu().numpy()[rows],
                      codes.coef.cpu().numpy()[rows], codes.res_energy.cpu().numpy()[rows])
    rep.assert_ok()

    rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    out = gpu_ctx.iterate(Yg, D1g, D2g, 6, rmse_out=rmse)
    assert gpu_ctx.status() == 0
    D1n, D2n = D1g.cpu().numpy().astype(np.float64), D2g.cpu().numpy().astype(np.float64)
    assert np.allclose(np.linalg.norm(D1n, axis=0), 1.0, atol=1e-5)
    assert np.allclose(np.linalg.norm(D2n, axis=0), 1.0, atol=1e-5)
    sup = out.support.cpu().numpy().astype(np.int64)
    cf = out.coef.cpu().numpy().astype(np.float64)
    explicit = oracle.rmse(Y, D1n, D2n, sup, cf)
    assert abs(rmse.cpu().numpy()[1] - explicit) / explicit < 2e-4


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_signal(gpu_ctx):
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Y = np.zeros((0, 8, 8))
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    out = gpu_ctx.sparse_code(Yg, D1g, D2g, 4)
    assert out.support.shape == (0, 4)
    Y1 = np.random.default_rng(3).standard_normal((1, 8, 8))
    check_code(gpu_ctx, Y1, D1, D2, 4)


def test_nonfinite_signal_flagged(gpu_ctx):
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((100, 8, 8))
    Y[17, 3, 2] = np.nan
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    out = gpu_ctx.sparse_code(Yg, D1g, D2g, 4)
    assert gpu_ctx.status() == -3          # SDL_ERR_NONFINITE, then cleared
    assert gpu_ctx.status() == 0
    nnz = out.nnz.cpu().numpy()
    assert nnz[17] == 0 and np.all(nnz[np.arange(100) != 17] == 4)


def test_zero_signal_gets_empty_code(gpu_ctx):
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Y = np.zeros((3, 8, 8))
    Y[1] = np.random.default_rng(2).standard_normal((8, 8))
    _, _, nnz, _ = run_code(gpu_ctx, Y, D1, D2, 4)
    assert list(nnz) == [0, 4, 0]


def test_host_argument_errors(gpu_ctx):
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Y = np.random.default_rng(1).standard_normal((10, 8, 8))
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    with pytest.raises(sdl.SDLError) as e:
        gpu_ctx.sparse_code(Yg, D1g, D2g, 65)
    assert e.value.code in (-1, -7)
    Dbig = sdl.dictionary(torch.randn(8, 300, device="cuda:0"))
    with pytest.raises(sdl.SDLError) as e:
        gpu_ctx.sparse_code(Yg, Dbig, D2g, 4)
    assert e.value.code == -7
    with pytest.raises(ValueError):
        gpu_ctx.sparse_code(Yg.contiguous(), D1g, D2g, 4)   # wrong memory layout


def test_bounded_wait_times_out_and_context_survives(gpu_ctx):
    """A wait on an mbarrier that nothing completes runs out after its cycle
    bound (here 2^24 cycles, about 8 ms) and records SDL_ERR_TIMEOUT; the
    next status read is clean and the context still codes correctly."""
    gpu_ctx.selftest_timeout(1 << 24)
    assert sdl.ERRORS[gpu_ctx.status()] == "SDL_ERR_TIMEOUT"
    assert gpu_ctx.status() == 0
    Y, _, _, _, _ = synth.kron_model(512, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    check_code(gpu_ctx, Y, D1, D2, 4)


# ------------------------------------------------------------- every tiling
@pytest.mark.parametrize("p1,n1,s,N", [(8, 16, 4, 4099), (12, 24, 6, 3001), (16, 32, 8, 1501)])
def test_every_tiling_gives_identical_codes_and_matches_oracle(gpu_ctx, p1, n1, s, N):
    """Pin each compiled tiling in turn (one and two signals per warp, both lane
    grids, 1 or 2 CTAs per SM): the codes are bit-identical across tilings,
    with and without the error-driven stop, and one Algorithm-1 iteration
    matches the oracle with each, with and without the stop.  About 40 % of
    the signals are halved, so that with the stop they start within the error
    target and take no atom: neighbours (the two halves of a warp) then mix
    signals that skip their correlations with signals that code."""
    tilings = sdl.tilings(p1, p1, n1, n1, s)
    assert len(tilings) >= 2
    rng = np.random.default_rng(77 + p1)
    Y = rng.standard_normal((N, p1, p1))
    Y[rng.random(N) < 0.4] *= 0.5           # ||Y|| about 0.5 p: below eps
    D1, D2 = synth.init_dictionaries(p1, p1, n1, n1, seed=1)
    eps = 0.8 * np.sqrt(p1 * p1)            # the others stop before or at s picks
    ref = oracle.omp2d(Y, D1, D2, s)
    ref_eps = oracle.omp2d(Y, D1, D2, s, eps=eps)
    skipped = ref_eps.nnz == 0
    assert 0.3 * N < skipped.sum() < 0.5 * N
    it_ref = oracle.iterate(Y, D1, D2, s)
    it_ref_eps = oracle.iterate(Y, D1, D2, s, eps=eps)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    first = first_eps = None
    try:
        for t in tilings:
            for cps in (1, 2):
                gpu_ctx.set_tiling(p1, p1, n1, n1, s, t, cps)
                for e, r in ((0.0, ref), (eps, ref_eps)):
                    out = gpu_ctx.sparse_code(Yg, D1g, D2g, s, eps=e)
                    assert gpu_ctx.status() == 0
                    got = (out.support.cpu(), out.coef.cpu(), out.nnz.cpu(), out.res_energy.cpu())
                    if e == 0.0:
                        first = first or got
                        base = first
                    else:
                        first_eps = first_eps or got
                        base = first_eps
                    for x, y in zip(got, base):
                        assert torch.equal(x, y), (t, cps, e)
                    if got is base:   # identical codes: the oracle judges them once
                        check_codes(Y, D1, D2, s, got[0].numpy(), got[2].numpy(), got[1].numpy(),
                                    got[3].numpy(), eps=(e or None), ref=r).assert_ok()
            for e, r in ((0.0, it_ref), (eps, it_ref_eps)):
                iterate_and_check(gpu_ctx, Y, D1, D2, s, eps=(e or None), ref=r,
                                  Ygpu=(Yg, D1g, D2g))
    finally:
        gpu_ctx.set_tiling(p1, p1, n1, n1, s, -1)


def test_tune_tiling_pins_the_fastest(gpu_ctx):
    imgs = np.stack([synth.synthetic_image(300 + i) for i in range(2)])
    Y = synth.random_patches(imgs, 20_000, 12, seed=3)
    D1, D2 = synth.init_dictionaries(12, 12, 24, 24, seed=1)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    try:
        tid, log = gpu_ctx.tune_tiling(Yg, D1g, D2g, 6)
        assert tid in sdl.tilings(12, 12, 24, 24, 6)
        assert len(log) == 2 * len(sdl.tilings(12, 12, 24, 24, 6))
        assert min(log, key=lambda e: e["us"])["tiling"] == tid
        codes = gpu_ctx.sparse_code(Yg, D1g, D2g, 6)
        rows = np.arange(0, 20_000, 17)
        check_codes(Y[rows], D1, D2, 6, codes.support.cpu().numpy()[rows], codes.nnz.cpu().numpy()[rows],
                    codes.coef.cpu().numpy()[rows], codes.res_energy.cpu().numpy()[rows]).assert_ok()
    finally:
        gpu_ctx.set_tiling(12, 12, 24, 24, 6, -1)
    with pytest.raises(sdl.SDLError):
        gpu_ctx.set_tiling(12, 12, 24, 24, 6, sdl.tilings(8, 8, 16, 16, 4)[0])


@pytest.mark.parametrize("p1,n1,s", [(8, 16, 4), (12, 24, 6)])
def test_exact_tie_picks_the_smallest_pair_index_in_every_tiling(gpu_ctx, p1, n1, s):
    """D1 atoms 3 and 5 are the same column, so every pair (3, j) and (5, j)
    scores exactly the same in FP32 (the same FMA chains): the first pick must
    be the smaller q = 3 + n1 j (the oracle's rule), in every tiling, and the
    second copy never joins (its Cholesky pivot is zero)."""
    D1, D2 = synth.init_dictionaries(p1, p1, n1, n1, seed=1)
    D1[:, 5] = D1[:, 3]
    rng = np.random.default_rng(9)
    N = 300
    j = rng.integers(0, n1, N)
    Y = np.einsum("a,kb->kab", D1[:, 3], D2[:, j].T) * rng.uniform(1.0, 2.0, (N, 1, 1))
    Y += 1e-3 * rng.standard_normal(Y.shape)
    ref = oracle.omp2d(Y, D1, D2, s)
    assert np.all(ref.support[:, 0] == 3 + n1 * j)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    try:
        for t in sdl.tilings(p1, p1, n1, n1, s):
            gpu_ctx.set_tiling(p1, p1, n1, n1, s, t, 0)
            out = gpu_ctx.sparse_code(Yg, D1g, D2g, s)
            assert gpu_ctx.status() == 0
            sup = out.support.cpu().numpy()
            assert np.all(sup[:, 0] == 3 + n1 * j), t
            assert not np.any(sup == (5 + n1 * j)[:, None]), t     # the duplicate never joins
            rep = check_codes(Y, D1, D2, s, sup, out.nnz.cpu().numpy(), out.coef.cpu().numpy(),
                              out.res_energy.cpu().numpy(), ref=ref)
            rep.assert_ok()   # both sides resolve the planted exact ties to the smaller q
    finally:
        gpu_ctx.set_tiling(p1, p1, n1, n1, s, -1)
