"""Pins of the three-mode oracle (Remark 3) against the explicit Kronecker
dictionary, textbook 1D OMP, the two-mode oracle (p3 = n3 = 1), the
unfolding identity, least-squares optimality of each mode update and the
monotone iteration."""
import numpy as np
import pytest

import oracle
from oracle import tmod3
from paper_2007_03800_gb300 import synth


def rand_problem(rng, N, p, n, s):
    Ds = [synth.random_dictionary(pk, nk, rng) for pk, nk in zip(p, n)]
    Q = n[0] * n[1] * n[2]
    sup = np.stack([rng.choice(Q, s, replace=False) for _ in range(N)]).astype(np.int64)
    coef = rng.standard_normal((N, s))
    return Ds, sup, coef


def test_kronecker_identity_three_modes():
    rng = np.random.default_rng(71)
    p, n = (3, 4, 2), (5, 3, 4)
    Ds, sup, coef = rand_problem(rng, 10, p, n, 4)
    K = tmod3.kron3(*Ds)
    X = tmod3.densify3(sup, coef, *n)
    Y = tmod3.reconstruct3(*Ds, sup, coef)
    for k in range(10):
        assert np.allclose(Y[k].flatten(order="F"), K @ X[k].flatten(order="F"), atol=1e-12)
        # and the mode-k products written out
        Z = np.einsum("ai,bj,cl,ijl->abc", *Ds, X[k])
        assert np.allclose(Z, Y[k], atol=1e-12)


def test_unfolding_identity():
    """Y_(k) = D_k X_(k) (D_later (x) D_earlier)^T (Remark 3)."""
    rng = np.random.default_rng(72)
    p, n = (3, 4, 2), (5, 3, 4)
    Ds, sup, coef = rand_problem(rng, 1, p, n, 6)
    X = tmod3.densify3(sup, coef, *n)[0]
    Y = tmod3.reconstruct3(*Ds, sup, coef)[0]
    for k in range(3):
        o = [m for m in range(3) if m != k]
        T = np.kron(Ds[o[1]], Ds[o[0]])
        assert np.allclose(tmod3.unfold(Y, k), Ds[k] @ tmod3.unfold(X, k) @ T.T, atol=1e-12)


def test_omp3d_is_1d_omp_on_the_kronecker_dictionary():
    rng = np.random.default_rng(73)
    p, n, s = (3, 3, 2), (4, 3, 3), 4
    Ds = [synth.random_dictionary(pk, nk, rng) for pk, nk in zip(p, n)]
    Y = rng.standard_normal((20,) + p)
    res = tmod3.omp3d(Y, *Ds, s)
    K = tmod3.kron3(*Ds)
    for k in range(20):
        y = Y[k].flatten(order="F")
        S, r = [], y.copy()
        for _ in range(s):
            c = np.abs(K.T @ r)
            c[S] = -1.0
            S.append(int(np.argmax(c)))                   # first index on ties
            x, *_ = np.linalg.lstsq(K[:, S], y, rcond=None)
            r = y - K[:, S] @ x
        assert list(res.support[k]) == S
        assert np.allclose(res.coef[k], x, atol=1e-10)
        assert np.isclose(res.res_energy[k], r @ r, rtol=1e-9, atol=1e-12)


def test_two_mode_special_case():
    """p3 = n3 = 1, D3 = [[1]]: the three-mode coder and updates are the
    two-mode oracle's."""
    rng = np.random.default_rng(74)
    p1, p2, n1, n2, s = 4, 5, 6, 7, 3
    D1, D2 = synth.random_dictionary(p1, n1, rng), synth.random_dictionary(p2, n2, rng)
    D3 = np.ones((1, 1))
    Y2 = rng.standard_normal((40, p1, p2))
    Y3 = Y2[..., None]
    r3 = tmod3.omp3d(Y3, D1, D2, D3, s)
    r2 = oracle.omp2d(Y2, D1, D2, s)
    assert np.array_equal(r3.support, r2.support)
    assert np.allclose(r3.coef, r2.coef, atol=1e-12)
    u1 = tmod3.update_mode(Y3, [D1, D2, D3], r2.support, r2.coef, 0)
    v1 = oracle.update_D1(Y2, D1, D2, r2.support, r2.coef)
    assert np.allclose(u1.D, v1.D, atol=1e-10) and np.allclose(u1.coef, v1.coef, atol=1e-10)
    u2 = tmod3.update_mode(Y3, [D1, D2, D3], r2.support, r2.coef, 1)
    v2 = oracle.update_D2(Y2, D1, D2, r2.support, r2.coef)
    assert np.allclose(u2.D, v2.D, atol=1e-10) and np.allclose(u2.coef, v2.coef, atol=1e-10)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_mode_update_is_least_squares_optimum(k):
    rng = np.random.default_rng(75 + k)
    p, n, s, N = (3, 4, 3), (5, 4, 4), 4, 300
    Ds, sup, coef = rand_problem(rng, N, p, n, s)
    Y = rng.standard_normal((N,) + p)
    upd = tmod3.update_mode(Y, Ds, sup, coef, k)
    # rescaled codes with the normalised atom give the objective of D_k*
    base = upd.obj_after
    assert base <= upd.obj_before + 1e-9
    newDs = list(Ds)
    for _ in range(20):
        E = rng.standard_normal(Ds[k].shape) * 1e-3
        newDs[k] = upd.D + E
        assert tmod3.objective3(Y, *newDs, sup, upd.coef) >= base - 1e-9
    assert np.allclose(np.linalg.norm(upd.D, axis=0), 1.0)


def test_three_mode_updates_are_monotone():
    rng = np.random.default_rng(78)
    p, n, s, N = (3, 3, 4), (4, 4, 6), 3, 400
    Dt, sup, coef = rand_problem(rng, N, p, n, s)
    Y = tmod3.reconstruct3(*Dt, sup, coef) + 0.05 * rng.standard_normal((N,) + p)
    Ds = [synth.random_dictionary(pk, nk, rng) for pk, nk in zip(p, n)]
    first = None
    for _ in range(4):
        it = tmod3.iterate3(Y, *Ds, s)
        # every dictionary update lowers the objective of its codes
        for code, upd in it.passes:
            assert upd.obj_after <= upd.obj_before + 1e-9
            assert np.isclose(upd.obj_before, np.sum(code.res_energy), rtol=1e-9)
        first = it.rmse[0] if first is None else first
        Ds = it.D
    assert it.rmse[2] < first          # learning fits the planted model better


def test_replay3_of_own_sequence_reproduces_pursuit():
    Y, _, _, _ = synth.kron_model3(150, (4, 4, 4), (8, 8, 8), 4, 20.0, seed=81)
    rng = np.random.default_rng(1)
    Ds = [synth.random_dictionary(4, 8, rng) for _ in range(3)]
    ref = tmod3.omp3d(Y, *Ds, 4)
    rp = tmod3.omp3d_replay(Y, *Ds, ref.support, ref.nnz, 4)
    assert np.array_equal(rp.best_q, ref.support)
    assert np.array_equal(rp.pick, rp.best)
    assert np.allclose(rp.coef, ref.coef, rtol=1e-12, atol=1e-14)
    assert np.allclose(rp.res_energy, ref.res_energy, rtol=1e-12)


def test_replay3_forced_sequence_against_explicit_kronecker():
    """Forced triple sequences on 2x3x2 cubes against D3 (x) D2 (x) D1 written
    out: correlations of the explicit residual, lstsq fit, pivot^2 as the
    squared distance from the span of the selected atoms."""
    rng = np.random.default_rng(7)
    p, n, s, N = (2, 3, 2), (3, 4, 2), 4, 20
    Ds = [synth.random_dictionary(p[m], n[m], rng) for m in range(3)]
    Y = rng.standard_normal((N,) + p)
    Q = n[0] * n[1] * n[2]
    sup = np.stack([rng.choice(Q, s, replace=False) for _ in range(N)]).astype(np.int64)
    nnz = rng.integers(0, s + 1, N)
    sup[np.arange(s)[None, :] >= nnz[:, None]] = -1
    rp = tmod3.omp3d_replay(Y, *Ds, sup, nnz, s)
    K = tmod3.kron3(*Ds)
    for k in range(N):
        y = Y[k].flatten(order="F")
        S, r = [], y.copy()
        for t in range(min(nnz[k] + 1, s)):
            c = np.abs(K.T @ r)
            c[S] = -1.0
            assert np.isclose(rp.energy[k, t], r @ r, rtol=1e-10)
            assert np.isclose(rp.best[k, t], c.max(), rtol=1e-10, atol=1e-13)
            a = K[:, rp.best_q[k, t]]
            proj = K[:, S] @ np.linalg.lstsq(K[:, S], a, rcond=None)[0] if S else 0.0
            assert np.isclose(rp.best_piv2[k, t], np.sum((a - proj) ** 2), rtol=1e-8, atol=1e-12)
            if t == nnz[k]:
                break
            assert np.isclose(rp.pick[k, t], c[sup[k, t]], rtol=1e-10, atol=1e-13)
            S.append(int(sup[k, t]))
            x, *_ = np.linalg.lstsq(K[:, S], y, rcond=None)
            r = y - K[:, S] @ x
        if S:
            assert np.allclose(rp.coef[k, :len(S)], x, rtol=1e-9, atol=1e-11)
        assert np.isclose(rp.res_energy[k], r @ r, rtol=1e-10)
