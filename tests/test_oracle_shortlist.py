"""Pins of the learned coder's shortlist oracle (oracle/shortlist.py) against
things other than itself: the full pursuit when every pair is a candidate,
brute force over explicit Kronecker atoms, a hand-worked example, and rank
definitions checked pair by pair."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import shortlist as sl
from paper_2007_03800_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "omp2d_restricted_2x2.json")


def test_all_pairs_as_candidates_is_the_full_pursuit():
    Y, _, _, _, _ = synth.kron_model(300, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    full = oracle.omp2d(Y, D1, D2, 4)
    cand = np.tile(np.arange(256), (300, 1))
    res = sl.omp2d_restricted(Y, D1, D2, 4, cand)
    assert np.array_equal(res.support, full.support) and np.array_equal(res.nnz, full.nnz)
    assert np.allclose(res.coef, full.coef, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n1,n2,s,k", [(4, 4, 3, 6), (6, 4, 4, 9), (8, 8, 4, 12)])
def test_bruteforce_restricted_picks_on_4x4(n1, n2, s, k):
    """Every pick is the argmax of |D^T r| over the unselected candidates of
    the explicit D2 (x) D1 (first index on ties), the coefficients are lstsq
    on the picked columns, and a pick with zero score stops the signal."""
    rng = np.random.default_rng(500 + n1 + n2 + k)
    D1, D2 = synth.random_dictionary(4, n1, rng), synth.random_dictionary(4, n2, rng)
    N = 30
    Y = rng.standard_normal((N, 4, 4))
    cand = np.stack([rng.choice(n1 * n2, k, replace=False) for _ in range(N)])
    cand[:3, -2:] = -1                                   # shorter lists
    res = sl.omp2d_restricted(Y, D1, D2, s, cand)
    Dk = np.kron(D2, D1)
    for m in range(N):
        y = Y[m].flatten(order="F")
        c = [q for q in cand[m] if q >= 0]
        S, r = [], y.copy()
        for _ in range(s):
            sc = np.full(n1 * n2, -1.0)
            sc[c] = np.abs(Dk[:, c].T @ r)
            sc[S] = -1.0
            q = int(np.argmax(sc))
            if sc[q] <= 0:
                break
            S.append(q)
            x, *_ = np.linalg.lstsq(Dk[:, S], y, rcond=None)
            r = y - Dk[:, S] @ x
        assert list(res.support[m, :len(S)]) == S and res.nnz[m] == len(S)
        assert np.allclose(res.coef[m, :len(S)], x, rtol=1e-9, atol=1e-11)
        assert np.isclose(res.res_energy[m], r @ r, rtol=1e-10)


def test_hand_worked_restricted_example():
    """tests/golden/omp2d_restricted_2x2.json, derived by hand (D1 = D2 = I)."""
    g = json.load(open(GOLDEN))
    res = sl.omp2d_restricted(np.array(g["Y"])[None], np.array(g["D1"]), np.array(g["D2"]), g["s"],
                              np.array([g["candidates"]]))
    assert list(res.support[0]) == g["support"]
    assert np.allclose(res.coef[0], g["coef"], atol=1e-15)
    assert np.isclose(res.res_energy[0], g["res_energy"])
    full = oracle.omp2d(np.array(g["Y"])[None], np.array(g["D1"]), np.array(g["D2"]), g["s"])
    assert list(full.support[0]) == g["support_unrestricted"]


def test_key16_preserves_order():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(4000).astype(np.float32) * 10,
                        np.array([0.0, 1e-38, -1e-38, 3.4e38, -3.4e38], dtype=np.float32)])
    k = sl.key16(v)
    order = np.argsort(v, kind="stable")
    assert np.all(np.diff(k[order]) >= 0)                      # a < b  =>  key(a) <= key(b)
    assert sl.key16(np.float32(-0.0)) < sl.key16(np.float32(0.0))    # the two zeros are ordered
    # values that share their upper 16 bits share their key
    a = np.array([1.0], dtype=np.float32).view(np.uint32)
    b = (a | 0x0000FFFF).view(np.float32)
    assert sl.key16(np.float32(1.0)) == sl.key16(b)[0]


def test_shortlists_match_the_pairwise_rank():
    """The shortlist is the set of pairs that fewer than k1 pairs beat, the
    check set those beaten by k1 .. k2-1 pairs (p beats q when key16(p) >
    key16(q), or the keys are equal and p < q; NaN scores never rank), each
    set listed in increasing q and padded with -1."""
    rng = np.random.default_rng(4)
    N, Q, k1, k2 = 40, 96, 8, 24
    S = rng.standard_normal((N, Q)).astype(np.float32)
    S[:, 10] = S[:, 50]                                  # exact ties
    S[:, 20] = np.nextafter(S[:, 21], np.float32(np.inf))   # equal 16-bit keys, unequal floats
    S[0, :90] = np.nan                                   # fewer valid scores than k2
    S[1, 3:70] = np.nan                                  # fewer valid scores than k2, more than k1
    L = sl.shortlists(S, k1, k2)
    key = sl.key16(S)
    for n in range(N):
        valid = ~np.isnan(S[n])
        rank = np.array([(valid & ((key[n] > key[n, q]) | ((key[n] == key[n, q]) & (np.arange(Q) < q)))).sum()
                         for q in range(Q)])
        want1 = np.nonzero(valid & (rank < k1))[0]
        want2 = np.nonzero(valid & (rank >= k1) & (rank < k2))[0]
        assert list(L[n, :want1.size]) == list(want1) and np.all(L[n, want1.size:k1] == -1)
        assert list(L[n, k1:k1 + want2.size]) == list(want2) and np.all(L[n, k1 + want2.size:] == -1)
    assert np.all(L[0, 6:] == -1) and np.all(L[0, :6] >= 90)


def test_check_scores_pinned_by_explicit_residual():
    rng = np.random.default_rng(8)
    D1, D2 = synth.random_dictionary(4, 6, rng), synth.random_dictionary(4, 6, rng)
    Y = rng.standard_normal((12, 4, 4))
    cand = np.stack([rng.permutation(36) for _ in range(12)])
    res = sl.omp2d_restricted(Y, D1, D2, 3, cand[:, :8])
    maxe, worst = sl.check_scores(Y, D1, D2, res)
    Dk = np.kron(D2, D1)
    for m in range(12):
        y = Y[m].flatten(order="F")
        S = list(res.support[m, :res.nnz[m]])
        x = np.linalg.lstsq(Dk[:, S], y, rcond=None)[0]
        r = y - Dk[:, S] @ x
        others = [q for q in range(36) if q not in S]
        assert np.isclose(maxe[m], np.abs(Dk[:, others].T @ r).max(), rtol=1e-10)
        # the weakest greedy score: replay the picks and take each step's best
        rr, w = y.copy(), np.inf
        for t, q in enumerate(S):
            w = min(w, abs(Dk[:, q] @ rr))
            xs = np.linalg.lstsq(Dk[:, S[:t + 1]], y, rcond=None)[0]
            rr = y - Dk[:, S[:t + 1]] @ xs
        assert np.isclose(worst[m], w, rtol=1e-10)
