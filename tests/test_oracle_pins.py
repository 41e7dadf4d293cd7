"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the explicit
Kronecker dictionary (Sec. I identity), brute force on tiny inputs, an
independent OMP implementation, exact recovery guarantees, the closed forms
and optimality of Result 1 / Corollary 1, and the orthonormal and MOD special
cases.  A plausible slip in the oracle (wrong pair index, transposed
dictionary, dropped term, missing normalisation rescale, wrong tie rule)
fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2007_03800_gb300 import synth


def vec(M):
    """Column-order vectorisation (Sec. I)."""
    return M.reshape(M.shape[:-2] + (-1,), order="F") if M.ndim == 2 else \
        np.stack([m.flatten(order="F") for m in M])


def rand_sparse(rng, N, n1, n2, s):
    sup = np.stack([rng.choice(n1 * n2, s, replace=False) for _ in range(N)])
    coef = rng.standard_normal((N, s))
    return sup.astype(np.int64), coef


# ---------------------------------------------------------------- Sec. I
def test_kronecker_identity_residual():
    """||Y - D1 X D2^T||_F = ||vec Y - (D2 (x) D1) vec X||_2 with q = i + n1*j."""
    rng = np.random.default_rng(5)
    p1, p2, n1, n2, s, N = 3, 5, 4, 7, 3, 20
    D1, D2 = rng.standard_normal((p1, n1)), rng.standard_normal((p2, n2))
    Y = rng.standard_normal((N, p1, p2))
    sup, coef = rand_sparse(rng, N, n1, n2, s)
    Dk = np.kron(D2, D1)
    R = oracle.residual(Y, D1, D2, sup, coef)
    for k in range(N):
        x = np.zeros(n1 * n2)
        x[sup[k]] = coef[k]
        r = Y[k].flatten(order="F") - Dk @ x
        assert np.allclose(R[k].flatten(order="F"), r, rtol=0, atol=1e-12)
        # the dense code the oracle builds is the column-order un-vec of x
        X = oracle.densify(sup[k:k + 1], coef[k:k + 1], n1, n2)[0]
        assert np.array_equal(X.flatten(order="F"), x)
    assert np.isclose(oracle.objective(Y, D1, D2, sup, coef), np.sum(R * R), rtol=1e-14)


# ------------------------------------------------- 2D-OMP == 1D OMP on D2 (x) D1
def omp_1d_explicit(y, D, s):
    """Textbook 1D OMP on an explicit dictionary: argmax |D^T r| (first index on
    ties), coefficients by least squares (lstsq), residual formed explicitly."""
    S, r = [], y.copy()
    for _ in range(s):
        c = np.abs(D.T @ r)
        c[S] = -1.0
        S.append(int(np.argmax(c)))
        x, *_ = np.linalg.lstsq(D[:, S], y, rcond=None)
        r = y - D[:, S] @ x
    return S, x, r


@pytest.mark.parametrize("n1,n2,s", [(4, 4, 3), (6, 4, 4), (8, 8, 4), (4, 6, 2)])
def test_bruteforce_4x4_picks_and_coefficients(n1, n2, s):
    rng = np.random.default_rng(100 + n1 * 10 + n2)
    p1 = p2 = 4
    D1 = synth.random_dictionary(p1, n1, rng)
    D2 = synth.random_dictionary(p2, n2, rng)
    Y = rng.standard_normal((40, p1, p2))
    res = oracle.omp2d(Y, D1, D2, s)
    Dk = np.kron(D2, D1)
    for k in range(Y.shape[0]):
        y = Y[k].flatten(order="F")
        S, x, r = omp_1d_explicit(y, Dk, s)
        assert list(res.support[k]) == S                       # every greedy pick
        xp = np.linalg.pinv(Dk[:, S]) @ y                      # coefficients vs pseudoinverse
        assert np.allclose(res.coef[k], xp, rtol=1e-10, atol=1e-12)
        assert np.isclose(res.res_energy[k], r @ r, rtol=1e-10)


def test_omp_residual_not_below_best_subset():
    """The greedy s-term residual is never below the exhaustive best s-subset."""
    rng = np.random.default_rng(7)
    p1 = p2 = 4
    n1 = n2 = 4
    s = 2
    D1, D2 = synth.random_dictionary(p1, n1, rng), synth.random_dictionary(p2, n2, rng)
    Dk = np.kron(D2, D1)
    Y = rng.standard_normal((12, p1, p2))
    res = oracle.omp2d(Y, D1, D2, s)
    for k in range(Y.shape[0]):
        y = Y[k].flatten(order="F")
        best = min(np.sum((y - Dk[:, S] @ np.linalg.lstsq(Dk[:, S], y, rcond=None)[0]) ** 2)
                   for S in itertools.combinations(range(n1 * n2), s))
        assert res.res_energy[k] >= best * (1 - 1e-12)


def test_matches_independent_omp_library():
    """scikit-learn's orthogonal_mp (Cholesky-based, independent code) on the
    explicit D2 (x) D1 gives the same supports and coefficients."""
    sk = pytest.importorskip("sklearn.linear_model")
    rng = np.random.default_rng(3)
    p1, p2, n1, n2, s = 6, 5, 9, 8, 5
    D1, D2 = synth.random_dictionary(p1, n1, rng), synth.random_dictionary(p2, n2, rng)
    Y = rng.standard_normal((60, p1, p2))
    res = oracle.omp2d(Y, D1, D2, s)
    Dk = np.kron(D2, D1)
    Xs = sk.orthogonal_mp(Dk, vec(Y).T, n_nonzero_coefs=s)      # (n1n2, N)
    for k in range(Y.shape[0]):
        x = np.zeros(n1 * n2)
        x[res.support[k]] = res.coef[k]
        assert np.allclose(x, Xs[:, k], rtol=1e-9, atol=1e-11)


def test_tie_rule_smallest_pair_index():
    """Exactly equal scores: the pick is the smallest q = i + n1*j."""
    p = 4
    D1 = np.eye(p)
    D2 = np.eye(p)
    Y = np.zeros((1, p, p))
    Y[0, 2, 1] = 1.0     # q = 2 + 4*1 = 6
    Y[0, 1, 3] = -1.0    # q = 1 + 4*3 = 13
    Y[0, 3, 0] = 1.0     # q = 3
    res = oracle.omp2d(Y, D1, D2, 3)
    assert list(res.support[0]) == [3, 6, 13]


def test_error_bounded_stop_and_zero_score():
    rng = np.random.default_rng(11)
    D1, D2 = np.eye(4), np.eye(4)
    Y = np.zeros((2, 4, 4))
    Y[0, 0, 0], Y[0, 1, 1], Y[0, 2, 2] = 5.0, 2.0, 0.5
    Y[1] = rng.standard_normal((4, 4)) * 1e-3
    res = oracle.omp2d(Y, D1, D2, 4, eps=1.0)
    # signal 0: after 5 and 2 the residual is 0.5 <= 1 -> stop at 2 picks
    assert res.nnz[0] == 2 and list(res.support[0][:2]) == [0, 5]
    assert res.nnz[1] == 0 and np.all(res.support[1] == -1)
    # a zero signal: best score 0 -> no pick in fixed-s mode
    z = oracle.omp2d(np.zeros((1, 4, 4)), D1, D2, 3)
    assert z.nnz[0] == 0


# ------------------------------------------------------------ exact recovery
def test_exact_recovery_orthonormal_any_s():
    rng = np.random.default_rng(21)
    p = 6
    Q1, _ = np.linalg.qr(rng.standard_normal((p, p)))
    Q2, _ = np.linalg.qr(rng.standard_normal((p, p)))
    for s in (1, 4, 9):
        sup, coef = rand_sparse(rng, 50, p, p, s)
        coef = np.sign(coef) * (0.5 + np.abs(coef))
        Y = oracle.reconstruct(Q1, Q2, sup, coef)
        res = oracle.omp2d(Y, Q1, Q2, s)
        for k in range(50):
            order = np.argsort(res.support[k])
            want = np.argsort(sup[k])
            assert np.array_equal(res.support[k][order], sup[k][want])
            assert np.allclose(res.coef[k][order], coef[k][want], atol=1e-12)


def test_exact_recovery_low_coherence():
    """Unit-norm D = [I | H/sqrt(p)] has coherence mu = 1/sqrt(p); the pair
    dictionary has mu(D2 (x) D1) = max(mu1, mu2) and OMP recovers any s-sparse
    code with s < (1 + 1/mu)/2 (p = 16: s <= 2)."""
    import scipy.linalg
    p = 16
    D = np.hstack([np.eye(p), scipy.linalg.hadamard(p) / np.sqrt(p)])
    mu = np.max(np.abs(D.T @ D - np.eye(2 * p)))
    assert np.isclose(mu, 0.25)
    rng = np.random.default_rng(22)
    s = 2
    assert s < (1 + 1 / mu) / 2
    sup, coef = rand_sparse(rng, 200, 2 * p, 2 * p, s)
    Y = oracle.reconstruct(D, D, sup, coef)
    res = oracle.omp2d(Y, D, D, s)
    for k in range(200):
        assert set(res.support[k]) == set(sup[k])
        m = {q: c for q, c in zip(sup[k], coef[k])}
        assert np.allclose([m[q] for q in res.support[k]], res.coef[k], atol=1e-12)


def test_orthonormal_omp_is_hard_thresholding():
    """Remark 1: with orthonormal D1, D2 the s-sparse code is T_s(D1^T Y D2)."""
    rng = np.random.default_rng(23)
    p, s = 5, 7
    Q1, _ = np.linalg.qr(rng.standard_normal((p, p)))
    Q2, _ = np.linalg.qr(rng.standard_normal((p, p)))
    Y = rng.standard_normal((30, p, p))
    res = oracle.omp2d(Y, Q1, Q2, s)
    for k in range(30):
        C = (Q1.T @ Y[k] @ Q2).flatten(order="F")
        top = np.argsort(-np.abs(C), kind="stable")[:s]
        assert list(res.support[k]) == list(top)
        assert np.allclose(res.coef[k], C[top], atol=1e-12)


# -------------------------------------------------- Result 1 / Corollary 1
def _setup_update(seed=31, p1=6, p2=5, n1=9, n2=8, s=4, N=300):
    rng = np.random.default_rng(seed)
    D1, D2 = synth.random_dictionary(p1, n1, rng), synth.random_dictionary(p2, n2, rng)
    Y = rng.standard_normal((N, p1, p2))
    sup, coef = rand_sparse(rng, N, n1, n2, s)
    return Y, D1, D2, sup, coef


def test_D1_update_is_least_squares_optimum():
    """Corollary 1: D1* minimises sum ||Y_k - D1 T_k||^2 (zero gradient, any
    perturbation raises the objective); W1 leaves the objective unchanged."""
    Y, D1, D2, sup, coef = _setup_update()
    u = oracle.update_D1(Y, D1, D2, sup, coef)
    X = oracle.densify(sup, coef, D1.shape[1], D2.shape[1])
    T = X @ D2.T
    grad = np.einsum("kaq,kiq->ai", np.einsum("ai,kiq->kaq", u.Dstar, T) - Y, T)
    assert np.max(np.abs(grad)) < 1e-9 * np.max(np.abs(u.B))
    f = lambda D: np.sum((Y - np.einsum("ai,kiq->kaq", D, T)) ** 2)
    rng = np.random.default_rng(0)
    for _ in range(5):
        assert f(u.Dstar + 1e-3 * rng.standard_normal(u.Dstar.shape)) > f(u.Dstar)
    # normalisation: unit columns, objective unchanged, and monotone decrease
    assert np.allclose(np.linalg.norm(u.D, axis=0), 1.0, atol=1e-14)
    assert np.isclose(u.obj_after, f(u.Dstar), rtol=1e-12)
    assert u.obj_after <= u.obj_before * (1 + 1e-12)


def test_D2_update_is_least_squares_optimum():
    """Result 1 (optimal D2) with the same checks, on the Z_k = D1 X_k side."""
    Y, D1, D2, sup, coef = _setup_update(seed=32)
    u = oracle.update_D2(Y, D1, D2, sup, coef)
    X = oracle.densify(sup, coef, D1.shape[1], D2.shape[1])
    Z = D1 @ X
    f = lambda D: np.sum((Y - np.einsum("kaj,bj->kab", Z, D)) ** 2)
    grad = np.einsum("kab,kaj->bj", np.einsum("kaj,bj->kab", Z, u.Dstar) - Y, Z)
    assert np.max(np.abs(grad)) < 1e-9 * np.max(np.abs(u.B))
    rng = np.random.default_rng(1)
    for _ in range(5):
        assert f(u.Dstar + 1e-3 * rng.standard_normal(u.Dstar.shape)) > f(u.Dstar)
    assert np.allclose(np.linalg.norm(u.D, axis=0), 1.0, atol=1e-14)
    assert np.isclose(u.obj_after, f(u.Dstar), rtol=1e-12)
    assert u.obj_after <= u.obj_before * (1 + 1e-12)


def test_closed_form_optimal_value():
    """Result 1: the optimum equals C = tr(sum Y^T Y - (sum Y^T Z)(sum Z^T Z)^{-1}(sum Z^T Y))."""
    Y, D1, D2, sup, coef = _setup_update(seed=33)
    u = oracle.update_D2(Y, D1, D2, sup, coef)
    X = oracle.densify(sup, coef, D1.shape[1], D2.shape[1])
    Z = D1 @ X
    SYY = np.einsum("kab,kac->bc", Y, Y)
    SYZ = np.einsum("kab,kaj->bj", Y, Z)
    SZZ = np.einsum("kai,kaj->ij", Z, Z)
    C = np.trace(SYY - SYZ @ np.linalg.solve(SZZ, SYZ.T))
    assert np.isclose(u.obj_after, C, rtol=1e-10)
    v = oracle.update_D1(Y, D1, D2, sup, coef)
    T = X @ D2.T
    SYT = np.einsum("kap,kip->ai", Y, T)
    STT = np.einsum("kip,kjp->ij", T, T)
    C1 = np.sum(Y * Y) - np.trace(SYT @ np.linalg.solve(STT, SYT.T))
    assert np.isclose(v.obj_after, C1, rtol=1e-10)


def test_gram_shortcut():
    """Sec. III: Z_k^T Z_k = X_k^T G1 X_k and T_k T_k^T = X_k G2 X_k^T with
    G1 = D1^T D1, G2 = D2^T D2: the oracle's P and M equal the shortcut sums."""
    Y, D1, D2, sup, coef = _setup_update(seed=34)
    X = oracle.densify(sup, coef, D1.shape[1], D2.shape[1])
    G1, G2 = D1.T @ D1, D2.T @ D2
    P = np.einsum("kij,jl,kml->im", X, G2, X)
    M = np.einsum("kij,il,klm->jm", X, G1, X)
    assert np.allclose(oracle.update_D1(Y, D1, D2, sup, coef).P, P, rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.update_D2(Y, D1, D2, sup, coef).P, M, rtol=1e-12, atol=1e-12)


def test_rescale_keeps_reconstruction():
    """X <- W^{-1} X exactly compensates D <- D* W (Result 1 / Corollary 1)."""
    Y, D1, D2, sup, coef = _setup_update(seed=35)
    u = oracle.update_D1(Y, D1, D2, sup, coef)
    assert np.allclose(oracle.reconstruct(u.Dstar, D2, sup, coef),
                       oracle.reconstruct(u.D, D2, sup, u.coef), atol=1e-12)
    v = oracle.update_D2(Y, D1, D2, sup, coef)
    assert np.allclose(oracle.reconstruct(D1, v.Dstar, sup, coef),
                       oracle.reconstruct(D1, v.D, sup, v.coef), atol=1e-12)


def test_unused_atom_kept():
    Y, D1, D2, sup, coef = _setup_update(seed=36)
    n1 = D1.shape[1]
    sup = np.where(sup % n1 == 3, (sup // n1) * n1 + 4, sup)    # atom i=3 never used
    # duplicate pairs may appear after the remap; merge them by zeroing repeats
    for k in range(sup.shape[0]):
        _, first = np.unique(sup[k], return_index=True)
        keep = np.zeros(sup.shape[1], bool)
        keep[first] = True
        coef[k][~keep] = 0.0
    u = oracle.update_D1(Y, D1, D2, sup, coef)
    assert not u.used[3]
    assert np.array_equal(u.D[:, 3], D1[:, 3])
    assert u.obj_after <= u.obj_before * (1 + 1e-12)


def test_mod_special_case():
    """p2 = n2 = 1, D2 = [1]: 2D-OMP is 1D OMP and the D1 update is MOD,
    D = Y X^T (X X^T)^{-1} (then normalised)."""
    sk = pytest.importorskip("sklearn.linear_model")
    rng = np.random.default_rng(41)
    p, n, s, N = 8, 12, 3, 400
    D = synth.random_dictionary(p, n, rng)
    Ym = rng.standard_normal((p, N))
    Y = Ym.T[:, :, None]
    res = oracle.omp2d(Y, D, np.ones((1, 1)), s)
    Xs = sk.orthogonal_mp(D, Ym, n_nonzero_coefs=s)
    Xd = oracle.densify(res.support, res.coef, n, 1)[:, :, 0].T   # (n, N)
    assert np.allclose(Xd, Xs, atol=1e-10)
    u = oracle.update_D1(Y, D, np.ones((1, 1)), res.support, res.coef)
    Dmod = Ym @ Xd.T @ np.linalg.inv(Xd @ Xd.T)
    assert np.allclose(u.Dstar, Dmod, rtol=1e-9, atol=1e-11)


def test_iteration_monotone_updates():
    """Algorithm 1: each dictionary update does not increase Eq. (1) (2D-OMP
    itself may)."""
    Y, D1t, D2t, _, _ = synth.kron_model(800, 6, 6, 10, 10, 3, 20.0, seed=51)
    D1, D2 = synth.init_dictionaries(6, 6, 10, 10, seed=1)
    for _ in range(4):
        it = oracle.iterate(Y, D1, D2, 3)
        assert it.upd_a.obj_after <= it.upd_a.obj_before * (1 + 1e-12)
        assert it.upd_b.obj_after <= it.upd_b.obj_before * (1 + 1e-12)
        scale = Y.size
        assert np.isclose(it.rmse_after_D2, np.sqrt(it.upd_b.obj_after / scale))
        D1, D2 = it.D1, it.D2


def test_selected_pairs_never_reselected():
    """OMP's residual is orthogonal to the selected pairs, so the greedy step
    looks only at unselected pairs: with noiseless 2-sparse signals and s = 4
    the greedy loop keeps picking new pairs until every remaining score is
    exactly 0, and never re-picks a selected one (which the pivot rule would
    turn into an early stop)."""
    rng = np.random.default_rng(61)
    p1 = p2 = 4
    n1 = n2 = 6
    D1, D2 = synth.random_dictionary(p1, n1, rng), synth.random_dictionary(p2, n2, rng)
    sup, coef = rand_sparse(rng, 200, n1, n2, 2)
    Y = oracle.reconstruct(D1, D2, sup, coef)
    res = oracle.omp2d(Y, D1, D2, 4)
    assert np.sum(res.nnz == 4) > 150
    for k in range(200):
        t = res.nnz[k]
        # an early stop is only allowed when every remaining score is exactly 0
        assert t == 4 or (t >= 2 and res.top_val[k, t, 0] == 0.0)
        assert len(set(res.support[k][:t])) == t


# ------------------------------------------- forced-support replay (Sec. III step 1)
def test_replay_of_own_sequence_reproduces_omp():
    """Forced along the oracle's own picks, the replay takes the greedy rule's
    choice at every step (pick score = best score, best_q = the pick) and
    returns omp2d's coefficients and residual energies."""
    Y, _, _, _, _ = synth.kron_model(200, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    res = oracle.omp2d(Y, D1, D2, 4)
    rp = oracle.omp2d_replay(Y, D1, D2, res.support, res.nnz, 4)
    assert np.array_equal(rp.best_q, res.support)
    assert np.array_equal(rp.pick, rp.best)
    assert np.allclose(rp.coef, res.coef, rtol=1e-12, atol=1e-14)
    assert np.allclose(rp.res_energy, res.res_energy, rtol=1e-12)
    assert np.all(rp.pick_piv2 > oracle.PIVOT_REL * rp.pick_Att)


@pytest.mark.parametrize("n1,n2,s", [(4, 4, 3), (6, 4, 4), (8, 8, 5)])
def test_replay_forced_sequence_against_explicit_kronecker(n1, n2, s):
    """Arbitrary forced pick sequences (not the greedy ones, some ending
    early) on 4x4 signals, checked step by step against the explicit
    D2 (x) D1 (Sec. I): correlations of the explicit residual, the least-squares
    fit by lstsq on the explicit columns, pivot^2 as the squared distance of an
    atom from the span of the selected ones, and the residual energies."""
    rng = np.random.default_rng(400 + n1 + 10 * n2 + s)
    p1 = p2 = 4
    D1 = synth.random_dictionary(p1, n1, rng)
    D2 = synth.random_dictionary(p2, n2, rng)
    N = 25
    Y = rng.standard_normal((N, p1, p2))
    sup = np.stack([rng.choice(n1 * n2, s, replace=False) for _ in range(N)]).astype(np.int64)
    nnz = rng.integers(0, s + 1, N)
    sup[np.arange(s)[None, :] >= nnz[:, None]] = -1
    rp = oracle.omp2d_replay(Y, D1, D2, sup, nnz, s)
    Dk = np.kron(D2, D1)
    for k in range(N):
        y = Y[k].flatten(order="F")
        S = []
        r = y.copy()
        for t in range(min(nnz[k] + 1, s)):
            c = np.abs(Dk.T @ r)
            c[S] = -1.0
            assert np.isclose(rp.energy[k, t], r @ r, rtol=1e-10)
            assert np.isclose(rp.best[k, t], c.max(), rtol=1e-10, atol=1e-13)
            assert c[rp.best_q[k, t]] >= c.max() * (1 - 1e-12)
            # pivot^2 of the greedy choice: squared distance from span(S)
            a = Dk[:, rp.best_q[k, t]]
            proj = Dk[:, S] @ np.linalg.lstsq(Dk[:, S], a, rcond=None)[0] if S else 0.0
            assert np.isclose(rp.best_piv2[k, t], np.sum((a - proj) ** 2), rtol=1e-8, atol=1e-12)
            if t == nnz[k]:
                break
            q = int(sup[k, t])
            assert np.isclose(rp.pick[k, t], c[q], rtol=1e-10, atol=1e-13)
            S.append(q)
            x, *_ = np.linalg.lstsq(Dk[:, S], y, rcond=None)
            r = y - Dk[:, S] @ x
        # the final fit on the whole forced support
        if S:
            assert np.allclose(rp.coef[k, :len(S)], x, rtol=1e-9, atol=1e-11)
        assert np.all(rp.coef[k, len(S):] == 0.0)
        assert np.isclose(rp.res_energy[k], r @ r, rtol=1e-10)
        assert np.all(np.isnan(rp.energy[k, nnz[k] + 1:]))
