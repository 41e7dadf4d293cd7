"""Learned support proposal around 2D-OMP: labels from plain 2D-OMP, network
training on the GPU, and the learned coder measured against the plain coder.
Orchestration only; every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import sdl, synth


def kron_problem(ctx: sdl.Context, N: int, p: int, n: int, s: int, snr_db=20.0, seed=51,
                 dl_iterations=20, device="cuda:0"):
    """Signals of the separable generative model, dictionaries learned on them
    by plain DL (Algorithm 1, `dl_iterations` iterations from the seed-1
    initialisation), and the plain 2D-OMP codes (the training labels)."""
    Y, _, _, _, _ = synth.kron_model(N, p, p, n, n, s, snr_db, seed=seed)
    D1, D2 = synth.init_dictionaries(p, p, n, n, seed=1)
    Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device=device))
    D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=device))
    D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=device))
    codes = None
    for _ in range(dl_iterations):
        codes = ctx.iterate(Yg, D1g, D2g, s, out=codes)
    labels = ctx.sparse_code(Yg, D1g, D2g, s)
    ctx.check()
    return Yg, D1g, D2g, labels


def fresh_signals(N, p, n, s, snr_db=20.0, seed=52, device="cuda:0"):
    """Fresh signals from the same generative model (same true dictionaries)."""
    Y, _, _, _, _ = synth.kron_model(N, p, p, n, n, s, snr_db, seed=seed, dict_seeds=(51, 52))
    return sdl.signals(torch.tensor(Y, dtype=torch.float32, device=device))


def train(mlp: sdl.MLP, Y, labels: sdl.Codes, epochs=3, batch=4096, lr=2e-3, cosine=False,
          stream=None):
    """Adam over contiguous batches (the generator's signals are i.i.d.),
    optionally with a cosine decay of the step size over all steps.
    Returns the mean loss of every epoch."""
    import math
    N = Y.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device=Y.device)
    hist = []
    per_epoch = max((N - batch) // batch + 1, 0)
    total = max(epochs * per_epoch, 1)
    step = 0
    for _ in range(epochs):
        acc = torch.zeros(1, dtype=torch.float32, device=Y.device)
        nb = 0
        for a in range(0, N - batch + 1, batch):
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / total)) if cosine else lr
            mlp.train_step(Y[a:a + batch], labels.support[a:a + batch], lr_t, loss_out=loss,
                           stream=stream)
            acc += loss
            nb += 1
            step += 1
        hist.append((acc / max(nb, 1)).item())
    return hist


def compare(ctx: sdl.Context, mlp: sdl.MLP, Y, D1, D2, s, k=32, reps=3):
    """Learned coder vs plain coder on the same signals: RMSE of both (from
    the least-squares residual energies), fallback rate, share of signals
    with identical codes, the guard's view of its judging sample (learned and
    plain RMSE there, whether it re-coded everything), and device time of
    each (CUDA events, best of reps)."""
    N, p1, p2 = Y.shape

    def timed(fn):
        best = None
        out = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return out, best

    plain, t_plain = timed(lambda: ctx.sparse_code(Y, D1, D2, s))
    (learned, flags, nfb, guard), t_learned = timed(lambda: mlp.sparse_code(Y, D1, D2, s, k=k))
    ctx.check()
    scale = p1 * p2 * N
    rmse_plain = (plain.res_energy.double().sum() / scale).sqrt().item()
    rmse_learned = (learned.res_energy.double().sum() / scale).sqrt().item()
    same = (learned.support == plain.support).all(dim=1).double().mean().item()
    g = guard.tolist()
    return dict(rmse_plain=rmse_plain, rmse_learned=rmse_learned,
                rmse_gap=rmse_learned / rmse_plain - 1.0,
                fallback_rate=nfb.item() / N, identical_codes=same,
                guard_sample_rmse_learned=g[0], guard_sample_rmse_plain=g[1],
                guard_sample_gap=g[0] / g[1] - 1.0 if g[1] > 0 else 0.0, guard_tripped=bool(g[2]),
                ms_plain=t_plain, ms_learned=t_learned, speedup=t_plain / t_learned, N=N)
