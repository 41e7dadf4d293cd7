"""Learned support proposal: gradients of the GPU training kernels against
the FP64 oracle, and what the trained network gains over an untrained one."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2007_03800_gb300 import learned, sdl, synth
from parity import to_gpu_problem

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def test_gradients_match_oracle(gpu_ctx):
    p, n, s, H, B = 8, 16, 4, 64, 128
    Y, D1, D2, _, _ = synth.kron_model(B, p, p, n, n, s, 20.0, seed=71)
    labels = oracle.omp2d(Y, D1, D2, s).support
    rng = np.random.default_rng(72)
    W1 = rng.standard_normal((H, p * p)) * 0.2
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((n * n, H)) * 0.2
    b2 = rng.standard_normal(n * n) * 0.1
    net = sdl.MLP(gpu_ctx, p, p, n, n, hidden=H, max_batch=B)
    net.set_weights(W1, b1, W2, b2)
    Yg, _, _ = to_gpu_problem(Y, D1, D2)
    sup = torch.tensor(labels, dtype=torch.int32, device="cuda:0")
    loss, g = net.gradients(Yg, sup)
    # oracle on the same BF16-rounded inputs and weights
    X = bf16(omlp.inputs(Y))
    T = omlp.targets(labels, n * n)
    ref_loss, ref = omlp.loss_and_grads(X, T, bf16(W1), b1, bf16(W2), b2)
    assert abs(loss - ref_loss) / ref_loss < 1e-2
    for name in ("W1", "b1", "W2", "b2"):
        err = np.linalg.norm(g[name] - ref[name]) / np.linalg.norm(ref[name])
        assert err < 3e-2, (name, err)
    net.close()


def test_training_lowers_loss_and_beats_untrained_network(gpu_ctx):
    """8x8 Kronecker workload: train on 64k OMP-labelled signals, then code
    16k fresh ones.  The trained network's shortlists must reproduce the
    plain codes far more often than an untrained network's, fall back less,
    and keep the RMSE within 1 % of the plain coder."""
    p, n, s = 8, 16, 4
    Y, D1g, D2g, labels = learned.kron_problem(gpu_ctx, 65536, p, n, s, dl_iterations=5)
    Yt = learned.fresh_signals(16384, p, n, s)
    untrained = sdl.MLP(gpu_ctx, p, p, n, n, hidden=512, max_batch=4096)
    untrained.init(seed=3)
    before = learned.compare(gpu_ctx, untrained, Yt, D1g, D2g, s, reps=1)
    net = sdl.MLP(gpu_ctx, p, p, n, n, hidden=512, max_batch=4096)
    net.init(seed=3)
    hist = learned.train(net, Y, labels, epochs=4, batch=4096, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    after = learned.compare(gpu_ctx, net, Yt, D1g, D2g, s, reps=1)
    assert after["identical_codes"] > before["identical_codes"] + 0.3, (before, after)
    assert after["fallback_rate"] < before["fallback_rate"], (before, after)
    assert abs(after["rmse_gap"]) < 0.01, after
    net.close()
    untrained.close()
