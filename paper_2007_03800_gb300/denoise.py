"""Patch-based image denoising with separable dictionaries (Sec. IV), on the
batched GPU path: every stride-1 patch of each size is coded with
error-driven 2D-OMP (stop at ||R||_F <= 1.15 sigma p, at most s atoms), the
dictionaries of all patch sizes are learned together (one batch, one graph
per iteration), and each image is rebuilt by averaging the overlapping
reconstructions.  Orchestration only: every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import sdl, synth

DEFAULT_GROUPS = ((8, 16, 4), (12, 24, 6), (16, 32, 8))   # (p, n, s cap): D is p x n


def denoise(ctx: sdl.Context, noisy: torch.Tensor, sigma: float, groups=DEFAULT_GROUPS,
            iterations: int = 10, clean: torch.Tensor | None = None, dict_seed: int = 1,
            autotune: bool = True, graph: bool = True, stream=None, timing: bool = False):
    """Learn one dictionary pair per patch size on the noisy image itself and
    denoise with it.  Returns a dict with per-group images, PSNRs (if clean
    is given), the RMSE trajectory (iterations x 2*G) and the batch tuning;
    with timing, also the device time of each phase in ms (CUDA events on
    the stream): patch extraction, batch set-up (autotuning and graph
    capture), the learning iterations, the final coding pass, averaging."""
    H, W = noisy.shape
    evs = []

    def mark():
        if timing:
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream if stream is not None else torch.cuda.current_stream())
            evs.append(e)

    mark()
    specs, meta = [], []
    for p, n, s in groups:
        Y, means = sdl.extract_patches(noisy, p, stream=stream)
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=dict_seed)
        D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=noisy.device))
        D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=noisy.device))
        specs.append(dict(Y=Y, D1=D1g, D2=D2g, s=s, eps=1.15 * sigma * p))
        meta.append(dict(p=p, n=n, s=s, means=means))
    mark()
    batch = sdl.Batch(ctx, specs, autotune=autotune, graph=graph, stream=stream)
    rmse = torch.zeros(2 * len(specs), dtype=torch.float64, device=noisy.device)
    mark()
    traj = []
    for _ in range(iterations):
        batch.iterate(rmse_out=rmse, stream=stream)
        traj.append(rmse.clone())
    mark()
    batch.sparse_code(stream=stream)
    mark()
    out = dict(images=[], psnr=[], nnz_mean=[], nnz_hist=[], tuning=batch.tuning(),
               tuning_log=batch.tuning_log(), rmse=torch.stack(traj) if traj else None,
               dictionaries=[])
    for spec, m in zip(batch.groups, meta):
        img = sdl.patch_average(ctx, spec["codes"], m["means"], spec["D1"], spec["D2"], m["p"],
                                H, W, stream=stream)
        out["images"].append(img)
        out["nnz_mean"].append(spec["codes"].nnz.float().mean())
        out["nnz_hist"].append(torch.bincount(spec["codes"].nnz.long(), minlength=m["s"] + 1))
        out["dictionaries"].append((spec["D1"], spec["D2"]))
        if clean is not None:
            out["psnr"].append(sdl.psnr(img, clean, stream=stream))
    mark()
    if timing:
        evs[-1].synchronize()
        names = ("extract", "setup", "iterations", "final_code", "average")
        out["ms_phases"] = {k: evs[i].elapsed_time(evs[i + 1]) for i, k in enumerate(names)}
    batch.close()
    return out


def orthonormal_start(p: int, seed: int):
    """Q factor (signs fixed by R's diagonal) of a seeded p x p N(0,1) matrix."""
    import numpy as np
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((p, p)))
    return Q * np.sign(np.diag(R))


def table3_case(ctx: sdl.Context, clean: torch.Tensor, noisy: torch.Tensor, sigma: float,
                variant: str = "general", p: int = 8, n: int = 16, train_patches: int = 4000,
                train_s: int = 6, iterations: int = 50, patch_seed: int = 0, dict_seed: int = 1,
                stream=None):
    """The denoising protocol of Table III (Sec. IV) on the GPU: dictionaries
    learned on `train_patches` mean-removed p x p patches of the noisy image at
    seeded positions with sparsity `train_s` (general: D1, D2 p x n by
    Algorithm 1; ortho: p x p orthonormal by Algorithm 1 - Orthonormal), then
    every overlapping patch coded error-driven (eps = 1.15 sigma p, at most p/2
    atoms), the image rebuilt by averaging, and PSNR / SSIM against `clean`."""
    import numpy as np
    H, W = noisy.shape
    dev = noisy.device
    imgs = noisy.detach().cpu().numpy()[None].astype(np.float64)
    Ytr = synth.random_patches(imgs, train_patches, p, seed=patch_seed)
    Yg = sdl.signals(torch.tensor(Ytr, dtype=torch.float32, device=dev))
    if variant == "general":
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=dict_seed)
    elif variant == "ortho":
        D1, D2 = orthonormal_start(p, dict_seed), orthonormal_start(p, dict_seed + 1)
    else:
        raise ValueError(variant)
    D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=dev))
    D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=dev))
    codes = None
    for _ in range(iterations):
        if variant == "general":
            codes = ctx.iterate(Yg, D1g, D2g, train_s, out=codes, stream=stream)
        else:
            codes = ctx.ortho_iterate(Yg, D1g, D2g, train_s, out=codes, stream=stream)
    Y, means = sdl.extract_patches(noisy, p, stream=stream)
    eps = 1.15 * sigma * p
    if variant == "general":
        code = ctx.sparse_code(Y, D1g, D2g, p // 2, eps=eps, stream=stream)
    else:
        code = ctx.ortho_sparse_code(Y, D1g, D2g, p // 2, eps=eps, stream=stream)
    img = sdl.patch_average(ctx, code, means, D1g, D2g, p, H, W, stream=stream)
    return dict(image=img, psnr=sdl.psnr(img, clean, stream=stream),
                ssim=sdl.ssim(ctx, img, clean, stream=stream),
                nnz_mean=code.nnz.float().mean(), dictionaries=(D1g, D2g))
