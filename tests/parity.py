"""Comparison helpers between the CUDA path and the FP64 oracle.

Supports: element-by-element equality of the pick sequences, except where the
oracle itself shows a tie at the first differing step: the GPU's pick must
then be among the oracle's top candidates with a score within TIE_REL of the
best (the FP32 kernel and the FP64 oracle can order near-equal scores
differently).  Signals with such a tie are counted and excluded from the
coefficient comparison, since their later picks legitimately diverge.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2007_03800_gb300 import sdl

TIE_REL = 1e-6       # relative score window of an argmax tie
COEF_RTOL = 1e-4     # per-signal ||x_gpu - x_ref|| / ||x_ref||
DICT_RTOL = 1e-4     # max |D_gpu - D_ref| (unit-norm columns)
RMSE_RTOL = 1e-4


def to_gpu_problem(Y, D1, D2, device="cuda:0"):
    Yg = sdl.signals(torch.tensor(np.asarray(Y), dtype=torch.float32, device=device))
    D1g = sdl.dictionary(torch.tensor(np.asarray(D1), dtype=torch.float32, device=device))
    D2g = sdl.dictionary(torch.tensor(np.asarray(D2), dtype=torch.float32, device=device))
    return Yg, D1g, D2g


def codes_from_oracle(support, coef, device="cuda:0"):
    sup = torch.tensor(np.asarray(support), dtype=torch.int32, device=device)
    cf = torch.tensor(np.where(np.asarray(support) >= 0, coef, 0.0), dtype=torch.float32, device=device)
    nnz = (sup >= 0).sum(dim=1).to(torch.int32)
    return sdl.Codes(sup, cf, nnz)


class SupportReport:
    def __init__(self, n, exact, ties, bad, bad_examples):
        self.n, self.exact, self.ties, self.bad = n, exact, ties, bad
        self.bad_examples = bad_examples

    def __repr__(self):
        return (f"SupportReport(n={self.n}, exact={self.exact}, ties={self.ties}, "
                f"bad={self.bad}, examples={self.bad_examples[:3]})")


def compare_supports(gpu_sup, gpu_nnz, ref, tie_rel=TIE_REL, eps=None, Y=None):
    """Classify every signal: identical pick sequence, a tie at the first
    difference (allowed, counted), or a mismatch (a failure)."""
    gpu_sup = np.asarray(gpu_sup)
    gpu_nnz = np.asarray(gpu_nnz)
    same = np.all(gpu_sup == ref.support, axis=1) & (gpu_nnz == ref.nnz)
    exact = same.copy()
    ties = np.zeros_like(same)
    bad = []
    for k in np.nonzero(~same)[0]:
        diff = np.nonzero(gpu_sup[k] != ref.support[k])[0]
        t = int(diff[0]) if diff.size else int(min(gpu_nnz[k], ref.nnz[k]))
        g = gpu_sup[k, t] if t < gpu_sup.shape[1] else -1
        if g >= 0 and ref.support[k, t] >= 0:
            tq, tv = ref.top_q[k, t], ref.top_val[k, t]
            hit = np.nonzero(tq == g)[0]
            if hit.size and tv[hit[0]] >= (1.0 - tie_rel) * tv[0]:
                ties[k] = True
                continue
            bad.append((int(k), t, int(g), int(ref.support[k, t]),
                        float(tv[hit[0]] / tv[0]) if hit.size else None))
        else:
            # one side stopped where the other picked: allowed only at the
            # error-driven threshold (residual within the tie window of eps)
            if eps is not None:
                ties[k] = True
                continue
            bad.append((int(k), t, int(g), int(ref.support[k, t]), None))
    return SupportReport(len(same), int(exact.sum()), int(ties.sum()), len(bad), bad), exact


def coef_rel_error(gpu_coef, ref_coef, rows):
    g = np.asarray(gpu_coef, dtype=np.float64)[rows]
    r = np.asarray(ref_coef)[rows]
    num = np.linalg.norm(g - r, axis=1)
    den = np.maximum(np.linalg.norm(r, axis=1), 1e-30)
    return num / den
