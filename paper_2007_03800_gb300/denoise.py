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
            autotune: bool = True, graph: bool = True, stream=None):
    """Learn one dictionary pair per patch size on the noisy image itself and
    denoise with it.  Returns a dict with per-group images, PSNRs (if clean
    is given), the RMSE trajectory (iterations x 2*G) and the batch tuning."""
    H, W = noisy.shape
    specs, meta = [], []
    for p, n, s in groups:
        Y, means = sdl.extract_patches(noisy, p, stream=stream)
        D1, D2 = synth.init_dictionaries(p, p, n, n, seed=dict_seed)
        D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=noisy.device))
        D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=noisy.device))
        specs.append(dict(Y=Y, D1=D1g, D2=D2g, s=s, eps=1.15 * sigma * p))
        meta.append(dict(p=p, n=n, s=s, means=means))
    batch = sdl.Batch(ctx, specs, autotune=autotune, graph=graph, stream=stream)
    rmse = torch.zeros(2 * len(specs), dtype=torch.float32, device=noisy.device)
    traj = []
    for _ in range(iterations):
        batch.iterate(rmse_out=rmse, stream=stream)
        traj.append(rmse.clone())
    batch.sparse_code(stream=stream)
    out = dict(images=[], psnr=[], nnz_mean=[], tuning=batch.tuning(),
               rmse=torch.stack(traj) if traj else None, dictionaries=[])
    for spec, m in zip(batch.groups, meta):
        img = sdl.patch_average(ctx, spec["codes"], m["means"], spec["D1"], spec["D2"], m["p"],
                                H, W, stream=stream)
        out["images"].append(img)
        out["nnz_mean"].append(spec["codes"].nnz.float().mean())
        out["dictionaries"].append((spec["D1"], spec["D2"]))
        if clean is not None:
            out["psnr"].append(sdl.psnr(img, clean, stream=stream))
    batch.close()
    return out
