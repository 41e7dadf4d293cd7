"""Pins of the orthonormal-variant oracle (Remark 1) against facts the
mathematics fixes: thresholding is the best s-term code (brute force), it
equals the oracle's independent 2D-OMP for orthonormal dictionaries, the
Procrustes update beats every other orthonormal dictionary, it recovers a
planted orthonormal dictionary exactly, and the iteration never raises the
objective."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import ortho


def orth(rng, p):
    Q, R = np.linalg.qr(rng.standard_normal((p, p)))
    return Q * np.sign(np.diag(R))


def rand_sparse(rng, N, n1, n2, s):
    sup = np.stack([rng.choice(n1 * n2, s, replace=False) for _ in range(N)])
    return sup.astype(np.int64), rng.standard_normal((N, s))


def test_threshold_is_best_s_term_code_brute_force():
    """For orthonormal D1, D2 no other support of size s (with its LS
    coefficients) leaves a smaller residual than T_s(D1^T Y D2)."""
    rng = np.random.default_rng(41)
    p, s = 3, 2
    D1, D2 = orth(rng, p), orth(rng, p)
    Y = rng.standard_normal((8, p, p))
    sup, coef, res = ortho.threshold_code(Y, D1, D2, s)
    K = np.kron(D2, D1)
    for k in range(8):
        y = Y[k].flatten(order="F")
        best = np.inf
        for S in itertools.combinations(range(p * p), s):
            A = K[:, S]
            x, *_ = np.linalg.lstsq(A, y, rcond=None)
            best = min(best, np.sum((y - A @ x) ** 2))
        assert res[k] <= best + 1e-12
        # and its coefficients are the LS coefficients on its own support
        A = K[:, sup[k]]
        x, *_ = np.linalg.lstsq(A, y, rcond=None)
        assert np.allclose(coef[k], x, atol=1e-12)


def test_threshold_equals_omp_for_orthonormal_dictionaries():
    rng = np.random.default_rng(42)
    p, s = 6, 5
    D1, D2 = orth(rng, p), orth(rng, p)
    Y = rng.standard_normal((60, p, p))
    sup, coef, res = ortho.threshold_code(Y, D1, D2, s)
    omp = oracle.omp2d(Y, D1, D2, s)
    assert np.array_equal(sup, omp.support)
    assert np.allclose(coef, omp.coef, atol=1e-12)
    assert np.allclose(res, omp.res_energy, rtol=1e-10, atol=1e-12)


def test_threshold_skips_exact_zeros():
    D = np.eye(3)
    Y = np.zeros((2, 3, 3))
    Y[1, 0, 0] = 2.0                               # one nonzero entry
    sup, coef, res = ortho.threshold_code(Y, D, D, 2)
    assert list(sup[0]) == [-1, -1] and list(sup[1]) == [0, -1]
    assert list(coef[1]) == [2.0, 0.0] and res[1] == 0.0


def test_threshold_tie_goes_to_smaller_q():
    D = np.eye(2)
    Y = np.array([[[1.0, -1.0], [0.5, 1.0]]])     # |C| = 1 at q = 0, 2, 3
    sup, coef, _ = ortho.threshold_code(Y, D, D, 2)
    assert list(sup[0]) == [0, 2] and list(coef[0]) == [1.0, -1.0]


@pytest.mark.parametrize("side", [1, 2])
def test_procrustes_beats_every_other_orthonormal_dictionary(side):
    rng = np.random.default_rng(43 + side)
    p, s, N = 5, 3, 200
    D1, D2 = orth(rng, p), orth(rng, p)
    Y = rng.standard_normal((N, p, p))
    sup, coef = rand_sparse(rng, N, p, p, s)
    upd = (ortho.procrustes_D1 if side == 1 else ortho.procrustes_D2)(Y, D1, D2, sup, coef)
    D = upd.D
    assert np.allclose(D.T @ D, np.eye(p), atol=1e-12)

    def f(Dx):
        return oracle.objective(Y, Dx, D2, sup, coef) if side == 1 else \
            oracle.objective(Y, D1, Dx, sup, coef)

    best = f(D)
    for _ in range(50):
        assert best <= f(orth(rng, p)) + 1e-9
    # and every small rotation of it
    for _ in range(20):
        A = rng.standard_normal((p, p)) * 1e-3
        import scipy.linalg
        R = scipy.linalg.expm(A - A.T)
        assert best <= f(D @ R) + 1e-9


@pytest.mark.parametrize("side", [1, 2])
def test_procrustes_recovers_a_planted_dictionary(side):
    """Y_k = Q1 X_k Q2^T exactly with the true codes: B1 = Q1 sum X X^T
    (Q2 orthonormal), whose polar factor is Q1; mirrored for Q2."""
    rng = np.random.default_rng(45 + side)
    p, s, N = 6, 4, 400
    Q1, Q2 = orth(rng, p), orth(rng, p)
    sup, coef = rand_sparse(rng, N, p, p, s)
    Y = oracle.reconstruct(Q1, Q2, sup, coef)
    D0 = orth(rng, p)
    if side == 1:
        upd = ortho.procrustes_D1(Y, D0, Q2, sup, coef)
        assert np.allclose(upd.D, Q1, atol=1e-10)
    else:
        upd = ortho.procrustes_D2(Y, Q1, D0, sup, coef)
        assert np.allclose(upd.D, Q2, atol=1e-10)


def test_rank_deficient_procrustes_matrix_is_singular():
    rng = np.random.default_rng(47)
    p, N = 4, 50
    D1, D2 = orth(rng, p), orth(rng, p)
    Y = rng.standard_normal((N, p, p))
    # no code uses atom i = 3 of D1: column 3 of B1 is zero
    sup = np.stack([rng.choice([q for q in range(p * p) if q % p != 3], 3, replace=False)
                    for _ in range(N)]).astype(np.int64)
    coef = rng.standard_normal((N, 3))
    with pytest.raises(oracle.SingularError):
        ortho.procrustes_D1(Y, D1, D2, sup, coef)


def test_ortho_iteration_is_monotone_and_orthonormal():
    rng = np.random.default_rng(48)
    p, s, N = 6, 4, 500
    Q1, Q2 = orth(rng, p), orth(rng, p)
    sup, coef = rand_sparse(rng, N, p, p, s)
    Y = oracle.reconstruct(Q1, Q2, sup, coef) + 0.05 * rng.standard_normal((N, p, p))
    D1, D2 = orth(rng, p), orth(rng, p)
    prev = np.inf
    for _ in range(5):
        it = ortho.ortho_iterate(Y, D1, D2, s)
        # the D1 update cannot raise the objective of the first codes
        f_before = oracle.objective(Y, D1, D2, it.support_a, it.coef_a)
        f_after = oracle.objective(Y, it.D1, D2, it.support_a, it.coef_a)
        assert f_after <= f_before + 1e-9
        assert np.isclose(it.rmse_after_D1 ** 2 * Y.size, f_after, rtol=1e-10)
        assert it.rmse_after_D2 <= it.rmse_after_D1 + 1e-12
        assert it.rmse_after_D2 <= prev + 1e-12
        prev = it.rmse_after_D2
        for D in (it.D1, it.D2):
            assert np.allclose(D.T @ D, np.eye(p), atol=1e-12)
        D1, D2 = it.D1, it.D2


def test_error_driven_threshold_equals_error_driven_omp():
    """With an eps stop, thresholding on orthonormal dictionaries is error-driven
    OMP (the denoising coder of Sec. IV)."""
    rng = np.random.default_rng(49)
    p, s = 6, 5
    D1, D2 = orth(rng, p), orth(rng, p)
    Y = rng.standard_normal((80, p, p)) * rng.uniform(0.2, 2.0, (80, 1, 1))
    eps = 3.0
    sup, coef, res = ortho.threshold_code(Y, D1, D2, s, eps=eps)
    omp = oracle.omp2d(Y, D1, D2, s, eps=eps)
    assert np.array_equal(sup, omp.support)
    assert np.allclose(coef, omp.coef, atol=1e-12)
    assert np.allclose(res, omp.res_energy, rtol=1e-10, atol=1e-10)
    nnz = (sup >= 0).sum(axis=1)
    assert nnz.min() < nnz.max() <= s and np.any((nnz > 0) & (nnz < s))
