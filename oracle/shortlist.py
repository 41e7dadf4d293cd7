"""FP64 reference of the learned coder's shortlist steps (TEST INFRASTRUCTURE
ONLY, see the package docstring).  The paper has no learned proposal; these
rules define the extension's behaviour before its fallback to the full coder
(whose reference is sdl_oracle.omp2d, Sec. III step 1):

  shortlists        : per signal, rank the network's FP32 scores of the n1 n2
                      atom pairs by the order-preserving 16-bit key of each
                      score (its upper 16 bits after flipping negative values,
                      so that a larger float has a larger key), ties to the
                      smaller pair index q; the first k1 form the shortlist and
                      the next k2 - k1 the check set, each set listed in
                      increasing q (-1 where fewer scores exist; NaN scores
                      never rank).  Written as a stable sort, not as the
                      bisection the CUDA top-k uses.
  omp2d_restricted  : 2D-OMP whose greedy step only looks at the signal's
                      candidate pairs: argmax |C_q| over unselected candidates
                      (ties to the smallest q), the same full least-squares
                      re-fit, degenerate-pick and zero-score stops as omp2d.
  check_scores      : after the restricted pursuit, the largest |correlation|
                      of an unselected pair with the final residual, and the
                      weakest greedy score among the picks (a signal with s
                      picks is sent to the full coder when the first exceeds
                      0.7 x the second, or when it has non-finite data).
"""
from __future__ import annotations

import numpy as np

from .sdl_oracle import (PIVOT_REL, OMPResult, _cholesky_rows, _cholesky_solve, grams,
                         reconstruct)

__all__ = ["key16", "shortlists", "omp2d_restricted", "check_scores", "CHECK_MARGIN"]

CHECK_MARGIN = 0.7


def key16(scores) -> np.ndarray:
    """Order-preserving 16-bit key of FP32 values: for x >= 0 the bits with
    the sign bit set, for x < 0 the complemented bits, then the upper half."""
    u = np.asarray(scores, dtype=np.float32).view(np.uint32).astype(np.uint64)
    neg = (u & 0x80000000) != 0
    flipped = np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000)
    return (flipped >> 16).astype(np.int64)


def shortlists(scores, k1: int, k2: int) -> np.ndarray:
    """(N, k2) candidate lists: the k1 best pairs by (key16 descending, q
    ascending), then the next k2 - k1; each of the two sets in increasing q;
    NaN scores never rank."""
    scores = np.asarray(scores, dtype=np.float32)
    N, Q = scores.shape
    key = key16(scores)
    key = np.where(np.isnan(scores), -1, key)
    out = np.full((N, k2), -1, dtype=np.int64)
    q = np.arange(Q)
    for k in range(N):
        order = np.lexsort((q, -key[k]))          # last key primary: key desc, then q asc
        order = order[key[k][order] >= 0][:k2]
        first, rest = np.sort(order[:k1]), np.sort(order[k1:])
        out[k, :first.size] = first
        out[k, k1:k1 + rest.size] = rest
    return out


def omp2d_restricted(Y, D1, D2, s: int, cand, top_k: int = 4) -> OMPResult:
    """2D-OMP of every signal searching only its candidate pairs cand[k]
    (entries < 0 ignored).  Same re-fit and stopping rules as omp2d; top_q /
    top_val rank the unselected candidates at each step (for tie analysis)."""
    Y = np.asarray(Y, dtype=np.float64)
    D1 = np.asarray(D1, dtype=np.float64)
    D2 = np.asarray(D2, dtype=np.float64)
    cand = np.asarray(cand, dtype=np.int64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    nq = n1 * n2
    G1, G2 = grams(D1, D2)
    C0 = np.einsum("ai,kab,bj->kij", D1, Y, D2, optimize=True)
    allowed = np.zeros((N, nq), dtype=bool)
    rows = np.repeat(np.arange(N)[:, None], cand.shape[1], axis=1)
    allowed[rows[cand >= 0], cand[cand >= 0]] = True
    support = np.full((N, s), -1, dtype=np.int64)
    coef = np.zeros((N, s))
    nnz = np.zeros(N, dtype=np.int64)
    K = min(top_k, nq)
    top_q = np.full((N, s, K), -1, dtype=np.int64)
    top_val = np.full((N, s, K), np.nan)
    R = Y.copy()
    active = np.ones(N, dtype=bool)
    for t in range(s):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        C = np.einsum("ai,kab,bj->kij", D1, R[idx], D2, optimize=True)
        score = np.abs(C).transpose(0, 2, 1).reshape(idx.size, nq)   # column q = i + n1*j
        score[~allowed[idx]] = -1.0                                   # not a candidate
        r = np.arange(idx.size)
        for l in range(t):
            score[r, support[idx, l]] = -1.0                          # already selected
        order = np.lexsort((np.broadcast_to(np.arange(nq), score.shape), -score), axis=1)[:, :K]
        top_q[idx, t] = order
        top_val[idx, t] = np.take_along_axis(score, order, axis=1)
        q = order[:, 0]
        best = score[r, q]
        sup = np.concatenate([support[idx, :t], q[:, None]], axis=1)
        ii, jj = sup % n1, sup // n1
        A = G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]]
        L, piv2 = _cholesky_rows(A)
        accept = (best > 0) & (piv2 > PIVOT_REL * A[:, t, t])
        x = _cholesky_solve(L, C0[idx[:, None], ii, jj])
        acc = idx[accept]
        support[acc, t] = q[accept]
        coef[acc, :t + 1] = x[accept]
        nnz[acc] = t + 1
        R[acc] = Y[acc] - reconstruct(D1, D2, support[acc, :t + 1], coef[acc, :t + 1])
        active[idx[~accept]] = False
    res_energy = np.sum(R * R, axis=(1, 2))
    return OMPResult(support, coef, nnz, res_energy, top_q, top_val)


def check_scores(Y, D1, D2, res: OMPResult):
    """For each signal: the largest |<R, d1_i d2_j^T>| over the pairs it did
    not pick (R the final residual of `res`), and the weakest greedy score,
    i.e. the smallest best-score among its picks (top_val[:, t, 0], inf when
    it has none)."""
    Y = np.asarray(Y, dtype=np.float64)
    R = Y - reconstruct(D1, D2, res.support, res.coef)
    C = np.einsum("ai,kab,bj->kij", D1, R, D2, optimize=True)
    score = np.abs(C).transpose(0, 2, 1).reshape(Y.shape[0], -1)      # column q = i + n1*j
    rows = np.repeat(np.arange(Y.shape[0])[:, None], res.support.shape[1], axis=1)
    picked = res.support >= 0
    score[rows[picked], res.support[picked]] = 0.0
    worst = np.full(Y.shape[0], np.inf)
    for t in range(res.support.shape[1]):
        sel = res.support[:, t] >= 0
        worst = np.where(sel, np.minimum(worst, res.top_val[:, t, 0]), worst)
    return score.max(axis=1), worst
