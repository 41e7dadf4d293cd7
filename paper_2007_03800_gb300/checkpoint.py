"""Checkpoint / resume and per-iteration metrics for runs of Algorithm 1.

A checkpoint holds what the next iteration needs: D1 and D2 (as p x n
arrays), the number of iterations done, the run's configuration (a JSON
object: shapes, s, eps, seeds, ...) and its hash.  Every reduction of an
iteration runs in a fixed order, so a run resumed from a checkpoint follows
the trajectory of the uninterrupted run for the same launch configuration.
Checkpoints are written to a temporary file and renamed, so a crash leaves
either the old or the new one.

`learn` runs iterations through the library (`Context.iterate`) and writes one
JSON line per iteration: the RMSE after each dictionary update, the histogram
of code sizes, the device time and the throughput.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import sdl

__all__ = ["config_hash", "save", "load", "MetricsLog", "learn"]


def config_hash(config: dict) -> str:
    """Stable hash of a JSON-serialisable configuration (key order ignored)."""
    text = json.dumps(config, sort_keys=True, separators=(",", ":"))
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):                      # a torch tensor, on any device
        a = a.detach().cpu().numpy()
    return np.array(a, dtype=np.float32, copy=True)


def save(path: str, D1, D2, iteration: int, config: dict) -> None:
    """Write D1, D2 (p x n), the iteration count and the configuration."""
    tmp = f"{path}.tmp-{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, D1=_host(D1), D2=_host(D2), iteration=np.int64(iteration),
                 config=np.array(json.dumps(config, sort_keys=True)),
                 config_hash=np.array(config_hash(config)))
    os.replace(tmp, path)


def load(path: str, config: dict | None = None) -> dict:
    """Read a checkpoint; with `config`, refuse one written for another
    configuration (ValueError)."""
    with np.load(path, allow_pickle=False) as z:
        out = {"D1": z["D1"].copy(), "D2": z["D2"].copy(), "iteration": int(z["iteration"]),
               "config": json.loads(str(z["config"])), "config_hash": str(z["config_hash"])}
    if out["config_hash"] != config_hash(out["config"]):
        raise ValueError(f"{path}: configuration does not match its hash")
    if config is not None and config_hash(config) != out["config_hash"]:
        raise ValueError(f"{path}: written for another configuration")
    return out


class MetricsLog:
    """Append-only JSON-lines log, one object per call."""

    def __init__(self, path: str):
        self.path = path

    def log(self, **record) -> None:
        with open(self.path, "a") as f:
            f.write(json.dumps(record, sort_keys=True) + "\n")

    def read(self) -> list[dict]:
        if not os.path.exists(self.path):
            return []
        with open(self.path) as f:
            return [json.loads(line) for line in f if line.strip()]


def learn(ctx, Y, D1, D2, s: int, iterations: int, eps: float = 0.0, *, config: dict | None = None,
          checkpoint: str | None = None, every: int = 1, log: MetricsLog | None = None,
          start: int = 0):
    """Run Algorithm-1 iterations start+1 .. iterations on (Y, D1, D2) in place
    (device tensors in the library's layouts).  After every `every`
    iterations and after the last one, write `checkpoint` (if given); log one
    record per iteration (if `log` is given).  Returns the codes of the last
    iteration."""
    import torch

    if every < 1:
        raise ValueError("every must be at least 1")
    N = Y.shape[0]
    config = dict(config or {})
    rmse = torch.zeros(2, dtype=torch.float64, device=Y.device)
    codes = None
    for it in range(start + 1, iterations + 1):
        if Y.is_cuda:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            codes = ctx.iterate(Y, D1, D2, s, eps=eps, out=codes, rmse_out=rmse)
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
        else:   # a stand-in context (host tests)
            t0 = time.perf_counter()
            codes = ctx.iterate(Y, D1, D2, s, eps=eps, out=codes, rmse_out=rmse)
            ms = (time.perf_counter() - t0) * 1e3
        # a device-side error (non-finite data, a singular normal matrix, a
        # timed-out wait) leaves the dictionaries unusable: stop before this
        # iteration is logged or checkpointed
        code = ctx.status()
        if code != 0:
            raise sdl.SDLError(code, f"iteration {it}")
        if log is not None:
            hist = torch.bincount(codes.nnz.long(), minlength=s + 1).cpu().tolist()
            r = rmse.cpu().tolist()
            log.log(iteration=it, rmse_after_D1=r[0], rmse_after_D2=r[1], nnz_hist=hist,
                    ms=ms, signals_per_s=N / (ms / 1e3) if ms > 0 else None)
        if checkpoint and (it % every == 0 or it == iterations):
            save(checkpoint, D1, D2, it, config)
    return codes
