"""Batched problems (sdl_batch_*): groups of different shapes, sparsities and
stopping rules in one persistent launch per pass, with an autotuner and a
captured CUDA graph per iteration.  Each group must match the FP64 oracle
exactly as a stand-alone problem would."""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_03800_gb300 import sdl, synth
from parity import check_codes, check_iteration, to_gpu_problem

pytestmark = pytest.mark.gpu

SHAPES = [  # p, n, s, eps
    (8, 16, 4, 1.15 * 20.0 * 8),
    (12, 24, 6, 0.0),
    (16, 32, 8, 1.15 * 20.0 * 16),
]


def make_groups(seed=0, N=(3000, 2500, 1200)):
    img = synth.synthetic_image(300 + seed, size=160)
    noisy = img + np.random.default_rng(seed).normal(0, 20.0, img.shape)
    out = []
    for (p, n, s, eps), n_sig in zip(SHAPES, N):
        Y, _ = synth.all_patches(noisy, p)
        Y = Y[np.random.default_rng(seed + p).choice(Y.shape[0], n_sig, replace=False)]
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=1)
        out.append(dict(Y=Y, D1=D1, D2=D2, s=s, eps=eps))
    return out


def to_specs(groups):
    specs = []
    for g in groups:
        Yg, D1g, D2g = to_gpu_problem(g["Y"], g["D1"], g["D2"])
        specs.append(dict(Y=Yg, D1=D1g, D2=D2g, s=g["s"], eps=g["eps"]))
    return specs


def test_batch_sparse_code_matches_oracle_and_single_calls(gpu_ctx):
    groups = make_groups()
    specs = to_specs(groups)
    batch = sdl.Batch(gpu_ctx, specs, autotune=True, graph=False)
    batch.sparse_code()
    assert gpu_ctx.status() == 0
    for g, spec in zip(groups, batch.groups):
        eps = g["eps"] or None
        ref = oracle.omp2d(g["Y"], g["D1"], g["D2"], g["s"], eps=eps)
        codes = spec["codes"]
        check_codes(g["Y"], g["D1"], g["D2"], g["s"], codes.support.cpu().numpy(), codes.nnz.cpu().numpy(),
                    codes.coef.cpu().numpy(), eps=eps, ref=ref).assert_ok()
        # every lane tiling performs the same per-entry arithmetic: identical codes
        single = gpu_ctx.sparse_code(spec["Y"], spec["D1"], spec["D2"], spec["s"], eps=spec["eps"])
        assert torch.equal(single.support, codes.support)
        assert torch.equal(single.coef, codes.coef)
    tun = batch.tuning()
    assert len(tun) == 3 and all(t["ctas"] >= 1 and t["cost_us"] > 0 for t in tun)
    # a batch of the same groups reuses the context's result unless asked to re-time
    again = sdl.Batch(gpu_ctx, to_specs(groups), autotune=True, graph=False)
    assert again.tuning() == tun and again.tuning_log() == batch.tuning_log()
    again.close()
    fresh = sdl.Batch(gpu_ctx, to_specs(groups), autotune=True, graph=False, retune=True)
    assert [t["shape_id"] for t in fresh.tuning()] and len(fresh.tuning_log()) == len(batch.tuning_log())
    fresh.close()
    # the autotuner's log holds every timing it took; the chosen tiling is the fastest
    log = batch.tuning_log()
    for g, t in enumerate(tun):
        mine = [e for e in log if e["group"] == g]
        assert mine and min(e["cost_us"] for e in mine) == t["cost_us"]
        assert t["shape_id"] in {e["shape_id"] for e in mine}
    batch.close()


def test_batch_iterate_matches_oracle(gpu_ctx):
    groups = make_groups(seed=1)
    specs = to_specs(groups)
    batch = sdl.Batch(gpu_ctx, specs, autotune=True, graph=True)
    rmse = torch.zeros(6, dtype=torch.float64, device="cuda:0")
    batch.iterate(rmse_out=rmse)
    assert gpu_ctx.status() == 0
    r = rmse.cpu().numpy()
    for g, (grp, spec) in enumerate(zip(groups, batch.groups)):
        codes = spec["codes"]
        check_iteration(grp["Y"], grp["D1"], grp["D2"], grp["s"], codes.support.cpu().numpy(),
                        codes.nnz.cpu().numpy(), codes.coef.cpu().numpy(), spec["D1"].cpu().numpy(),
                        spec["D2"].cpu().numpy(), r[2 * g:2 * g + 2], eps=grp["eps"] or None)
    batch.close()


def test_graph_replay_equals_direct_launches(gpu_ctx):
    """The captured graph runs exactly the direct launch sequence: three
    iterations give bit-identical dictionaries, codes and RMSE."""
    groups = make_groups(seed=2, N=(1500, 1300, 700))
    results = []
    for graph in (False, True):
        specs = to_specs(groups)
        batch = sdl.Batch(gpu_ctx, specs, autotune=False, graph=graph)
        rmse = torch.zeros(6, dtype=torch.float64, device="cuda:0")
        for _ in range(3):
            batch.iterate(rmse_out=rmse)
        assert gpu_ctx.status() == 0
        results.append([(s["D1"].clone(), s["D2"].clone(), s["codes"].support.clone(),
                         s["codes"].coef.clone()) for s in batch.groups] + [rmse.clone()])
        batch.close()
    for a, b in zip(results[0][:-1], results[1][:-1]):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    assert torch.equal(results[0][-1], results[1][-1])


def test_batch_rejects_unsupported_shapes(gpu_ctx):
    """n2 = 256 is beyond every coder (compiled tilings and the generic kernel)."""
    Yg, D1g, D2g = to_gpu_problem(np.zeros((64, 16, 64)), *synth.init_dictionaries(16, 64, 32, 256))
    with pytest.raises(sdl.SDLError) as e:
        sdl.Batch(gpu_ctx, [dict(Y=Yg, D1=D1g, D2=D2g, s=10)])
    assert e.value.code == -7


def hsi_group(N=700, seed=37):
    """16 x 64 signals, D1 16 x 32, D2 64 x 128, s = 10: no compiled tiling.
    Signals of the separable model at those shapes (30 dB): its normal matrices
    are well conditioned, so the FP32 updates hold the 1e-4 dictionary bar (on
    the hyperspectral-shaped data few D2 atoms are used and cond(M) ~ 6e4)."""
    Y, *_ = synth.kron_model(N, 16, 64, 32, 128, 10, 30.0, seed=seed)
    D1, D2 = synth.init_dictionaries(16, 64, 32, 128, seed=1)
    return dict(Y=Y, D1=D1, D2=D2, s=10, eps=0.0)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_with_generic_shape_groups_matches_oracle(gpu_ctx, graph):
    """A group whose shape has no compiled tiling is coded by the generic
    kernel inside the batch iteration, beside compiled-tiling groups (and on
    its own): in both runs every group's iteration matches the oracle and
    the generic group's codes equal the per-call coder's; the compiled-tiling
    groups replay bit for bit, the generic group (whose teams add their partial
    sums with atomics, in no fixed order) to FP32 rounding."""
    for groups in (make_groups(seed=6, N=(1200, 1000, 600)) + [hsi_group()], [hsi_group(seed=38)]):
        G = len(groups)
        results = []
        for gr in (False, graph):
            specs = to_specs(groups)
            batch = sdl.Batch(gpu_ctx, specs, autotune=True, graph=gr)
            assert batch.tuning()[-1]["shape_id"] == -1 and batch.tuning()[-1]["ctas"] == 0
            rmse = torch.zeros(2 * G, dtype=torch.float64, device="cuda:0")
            batch.iterate(rmse_out=rmse)
            assert gpu_ctx.status() == 0
            results.append([(sp["D1"].clone(), sp["D2"].clone(), sp["codes"].support.clone(),
                             sp["codes"].coef.clone()) for sp in batch.groups] + [rmse.clone()])
            r = rmse.cpu().numpy()
            for g, (grp, sp) in enumerate(zip(groups, batch.groups)):
                codes = sp["codes"]
                check_iteration(grp["Y"], grp["D1"], grp["D2"], grp["s"],
                                codes.support.cpu().numpy(), codes.nnz.cpu().numpy(),
                                codes.coef.cpu().numpy(), sp["D1"].cpu().numpy(),
                                sp["D2"].cpu().numpy(), r[2 * g:2 * g + 2],
                                eps=grp["eps"] or None)
            # coding only, with the updated dictionaries: the per-call coder's codes
            batch.sparse_code()
            assert gpu_ctx.status() == 0
            sp = batch.groups[-1]
            single = gpu_ctx.sparse_code(sp["Y"], sp["D1"], sp["D2"], sp["s"])
            assert torch.equal(single.support, sp["codes"].support)
            assert torch.equal(single.coef, sp["codes"].coef)
            batch.close()
        for a, b in zip(results[0][:G - 1], results[1][:G - 1]):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
        assert torch.equal(results[0][-1][:2 * G - 2], results[1][-1][:2 * G - 2])
        for x, y in zip(results[0][G - 1][:2], results[1][G - 1][:2]):    # generic group's D1, D2
            assert (x - y).abs().max().item() < 1e-5
        assert torch.allclose(results[0][-1][2 * G - 2:], results[1][-1][2 * G - 2:], rtol=1e-6, atol=0)


@pytest.mark.parametrize("graph", [False, True])
def test_one_group_batch_runs_its_tiling_kernel_and_matches_oracle(gpu_ctx, graph):
    """A one-group batch codes with its tiling's own kernel (no multi-problem
    launch): one iteration matches the oracle, and the graph replays the
    direct launches bit for bit."""
    g = make_groups(seed=5)[1]
    ref = oracle.iterate(g["Y"], g["D1"], g["D2"], g["s"], eps=g["eps"] or None)
    results = []
    for gr in (False, graph):
        spec = to_specs([g])
        batch = sdl.Batch(gpu_ctx, spec, autotune=False, graph=gr)
        rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
        batch.iterate(rmse_out=rmse)
        assert gpu_ctx.status() == 0
        s = batch.groups[0]
        check_iteration(g["Y"], g["D1"], g["D2"], g["s"], s["codes"].support.cpu().numpy(),
                        s["codes"].nnz.cpu().numpy(), s["codes"].coef.cpu().numpy(), s["D1"].cpu().numpy(),
                        s["D2"].cpu().numpy(), rmse.cpu().numpy(), eps=g["eps"] or None, ref=ref)
        results.append((s["D1"].clone(), s["D2"].clone(), s["codes"].coef.clone(), rmse.clone()))
        batch.close()
    for x, y in zip(*results):
        assert torch.equal(x, y)


def test_one_group_batch_equals_the_per_call_path_at_full_size(gpu_ctx):
    """The benchmark workload (200 000 12x12 patches, D 12x24, s = 6) through a
    one-group autotuned, graph-replayed batch gives, bit for bit, the
    dictionaries and codes of the per-call iteration pinned to the same tiling
    and CTAs per SM; the per-call path is checked against the oracle at this
    size in test_gpu_parity.py."""
    imgs = np.stack([synth.synthetic_image(100 + i) for i in range(8)])
    Y = synth.random_patches(imgs, 200_000, 12, seed=5)
    D1, D2 = synth.init_dictionaries(12, 12, 24, 24, seed=1)
    Yg, D1g, D2g = to_gpu_problem(Y, D1, D2)
    D1b, D2b = D1g.clone(), D2g.clone()
    batch = sdl.Batch(gpu_ctx, [dict(Y=Yg, D1=D1b, D2=D2b, s=6, eps=0.0)], autotune=True, graph=True)
    rmse_b = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    batch.iterate(rmse_out=rmse_b)
    assert gpu_ctx.status() == 0
    t = batch.tuning()[0]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert t["ctas"] % sms == 0
    try:
        gpu_ctx.set_tiling(12, 12, 24, 24, 6, t["shape_id"], t["ctas"] // sms)
        rmse = torch.zeros(2, dtype=torch.float64, device="cuda:0")
        out = gpu_ctx.iterate(Yg, D1g, D2g, 6, rmse_out=rmse)
        assert gpu_ctx.status() == 0
    finally:
        gpu_ctx.set_tiling(12, 12, 24, 24, 6, -1)
    codes = batch.groups[0]["codes"]
    assert torch.equal(D1g, batch.groups[0]["D1"]) and torch.equal(D2g, batch.groups[0]["D2"])
    assert torch.equal(out.support, codes.support) and torch.equal(out.coef, codes.coef)
    # the objective change is an FP64 sum split over a different number of solve
    # threads: equal up to rounding
    assert torch.allclose(rmse, rmse_b, rtol=1e-9, atol=0)
    batch.close()
