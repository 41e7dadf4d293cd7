"""FP64 reference of the n-dimensional generalisation (Remark 3) for three
modes: signals Y_k of shape p1 x p2 x p3, dictionaries D1 (p1 x n1), D2
(p2 x n2), D3 (p3 x n3) with unit columns, and sparse cores X_k (n1 x n2 x n3)
with Y_k ~ X_k x_1 D1 x_2 D2 x_3 D3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What each routine follows:
  vec / Kronecker : vec(X x_1 D1 x_2 D2 x_3 D3) = (D3 (x) D2 (x) D1) vec(X) with
                    the column-order vec of Sec. I (first index fastest); atom
                    triple (i, j, l) <-> column q = i + n1 j + n1 n2 l
  omp3d           : greedy pursuit over atom triples (1D OMP on D3 (x) D2 (x) D1,
                    as 2D-OMP is on D2 (x) D1, Sec. II), full least-squares re-fit
                    after each pick, ties to the smallest q, the same degenerate-
                    pick rule as the 2-D oracle
  omp3d_replay    : the same pursuit forced along a given pick sequence (the
                    quantities of sdl_oracle.omp2d_replay, for atom triples)
  update_mode     : Remark 3 with X fixed: Y_(k) = D_k X_(k) T_k^T, T_k the
                    Kronecker product of the other dictionaries, so Corollary 1
                    gives D_k* = (sum Y_(k) T X_(k)^T)(sum X_(k) T^T T X_(k)^T)^{-1};
                    then the column normalisation W_k and X <- X W_k^{-1} along mode k
  iterate3        : code, D1 update, code, D2 update, code, D3 update (one coding
                    pass before each update, as Algorithm 1 does for two modes)

Readings: the mode order of the iteration and one
coding pass per update are the two-mode algorithm's pattern; unused atoms and
singular normal matrices follow the two-mode oracle.
"""
from __future__ import annotations

import numpy as np

from .sdl_oracle import (PIVOT_REL, ReplayResult, SingularError, _cholesky_rows, _cholesky_solve,
                         _solve_normal)

__all__ = ["kron3", "densify3", "reconstruct3", "objective3", "omp3d", "omp3d_replay",
           "update_mode", "iterate3", "unfold"]


def kron3(D1, D2, D3):
    """The Kronecker dictionary D3 (x) D2 (x) D1 (column q = i + n1 j + n1 n2 l)."""
    return np.kron(D3, np.kron(D2, D1))


def densify3(support, coef, n1, n2, n3):
    """Dense cores (N, n1, n2, n3) from (support, coef)."""
    N = support.shape[0]
    X = np.zeros((N, n1 * n2 * n3))
    valid = support >= 0
    rows = np.repeat(np.arange(N)[:, None], support.shape[1], axis=1)
    np.add.at(X, (rows[valid], support[valid]), coef[valid])
    return X.reshape(N, n3, n2, n1).transpose(0, 3, 2, 1)


def reconstruct3(D1, D2, D3, support, coef):
    n1, n2 = D1.shape[1], D2.shape[1]
    valid = support >= 0
    q = np.where(valid, support, 0)
    i, j, l = q % n1, (q // n1) % n2, q // (n1 * n2)
    x = np.where(valid, coef, 0.0)
    return np.einsum("km,akm,bkm,ckm->kabc", x, D1[:, i], D2[:, j], D3[:, l], optimize=True)


def objective3(Y, D1, D2, D3, support, coef) -> float:
    R = np.asarray(Y, dtype=np.float64) - reconstruct3(D1, D2, D3, support, coef)
    return float(np.sum(R * R))


def unfold(T, k: int):
    """Mode-k unfolding: rows = mode k, columns = the other modes in column
    order (the earlier mode fastest)."""
    T = np.moveaxis(T, k, 0)
    return T.reshape(T.shape[0], -1, order="F")


class OMP3Result:
    def __init__(self, support, coef, nnz, res_energy, top_q, top_val):
        self.support, self.coef, self.nnz = support, coef, nnz
        self.res_energy, self.top_q, self.top_val = res_energy, top_q, top_val


def omp3d(Y, D1, D2, D3, s: int, top_k: int = 4) -> OMP3Result:
    """Greedy pursuit over atom triples for every signal: explicit residual,
    correlations C = R x_1 D1^T x_2 D2^T x_3 D3^T, argmax |C| over unselected
    triples (ties -> smallest q), fresh Cholesky re-fit of all picks."""
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.shape[0]
    n1, n2, n3 = D1.shape[1], D2.shape[1], D3.shape[1]
    Q = n1 * n2 * n3
    G1, G2, G3 = D1.T @ D1, D2.T @ D2, D3.T @ D3
    C0 = np.einsum("ai,bj,cl,kabc->klji", D1, D2, D3, Y, optimize=True).reshape(N, Q)
    support = -np.ones((N, s), dtype=np.int64)
    coef = np.zeros((N, s))
    nnz = np.zeros(N, dtype=np.int64)
    top_q = -np.ones((N, s, top_k), dtype=np.int64)
    top_val = np.zeros((N, s, top_k))
    R = Y.copy()
    active = np.ones(N, dtype=bool)
    rows = np.arange(N)
    for t in range(s):
        C = np.einsum("ai,bj,cl,kabc->klji", D1, D2, D3, R, optimize=True).reshape(N, Q)
        score = np.abs(C)
        for m in range(t):
            score[rows, np.where(support[:, m] >= 0, support[:, m], 0)] = np.where(
                support[:, m] >= 0, -1.0, score[rows, 0])
        order = np.argsort(-score, axis=1, kind="stable")
        top_q[:, t, :] = order[:, :top_k]
        top_val[:, t, :] = np.take_along_axis(score, order[:, :top_k], axis=1)
        q = order[:, 0]
        best = score[rows, q]
        active &= best > 0.0
        cand = support.copy()
        cand[:, t] = q
        sel = cand[:, :t + 1]
        ii, jj, ll = sel % n1, (sel // n1) % n2, sel // (n1 * n2)
        A = (G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]] *
             G3[ll[:, :, None], ll[:, None, :]])
        Lc, piv2 = _cholesky_rows(A)
        ok = active & (piv2 > PIVOT_REL * A[:, t, t])
        b = np.take_along_axis(C0, sel, axis=1)
        x = _cholesky_solve(Lc, b)
        support[ok, t] = q[ok]
        coef[ok, :t + 1] = x[ok]
        nnz[ok] = t + 1
        active = ok
        R = Y - reconstruct3(D1, D2, D3, support, coef)
        if not active.any():
            break
    R = Y - reconstruct3(D1, D2, D3, support, coef)
    return OMP3Result(support, coef, nnz, np.einsum("kabc,kabc->k", R, R), top_q, top_val)


def _gram3(G1, G2, G3, sup, n1, n2):
    ii, jj, ll = sup % n1, (sup // n1) % n2, sup // (n1 * n2)
    return (G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]] *
            G3[ll[:, :, None], ll[:, None, :]])


def omp3d_replay(Y, D1, D2, D3, support, nnz, s: int) -> ReplayResult:
    """The pursuit of omp3d forced to take support[k, :nnz[k]] in that order
    (Remark 3's pursuit is 1D OMP on D3 (x) D2 (x) D1, Sec. II): at every step
    the residual of the previous fit gives the correlations, and the rule's
    own choice (max |C| over unselected triples, ties to the smallest q, with
    its pivot), the forced pick's score and pivot, and the residual energy are
    recorded; the coefficients are fitted on the forced support as omp3d does.
    Fields as sdl_oracle.ReplayResult."""
    Y = np.asarray(Y, dtype=np.float64)
    support = np.asarray(support, dtype=np.int64)
    nnz = np.asarray(nnz, dtype=np.int64)
    N = Y.shape[0]
    n1, n2, n3 = D1.shape[1], D2.shape[1], D3.shape[1]
    Q = n1 * n2 * n3
    G1, G2, G3 = D1.T @ D1, D2.T @ D2, D3.T @ D3
    C0 = np.einsum("ai,bj,cl,kabc->klji", D1, D2, D3, Y, optimize=True).reshape(N, Q)
    nan = lambda: np.full((N, s), np.nan)
    energy = np.full((N, s + 1), np.nan)
    best, best_piv2, best_Att = nan(), nan(), nan()
    pick, pick_piv2, pick_Att = nan(), nan(), nan()
    best_q = np.full((N, s), -1, dtype=np.int64)
    coef = np.zeros((N, s))
    R = Y.copy()
    for t in range(s + 1):
        live = np.nonzero(nnz >= t)[0]
        energy[live, t] = np.einsum("kabc,kabc->k", R[live], R[live])
        if t == s or live.size == 0:
            continue
        C = np.einsum("ai,bj,cl,kabc->klji", D1, D2, D3, R[live], optimize=True).reshape(live.size, Q)
        score = np.abs(C)
        rows = np.arange(live.size)
        prev = support[live, :t]
        for m in range(t):
            score[rows, prev[:, m]] = -1.0
        order = np.argsort(-score, axis=1, kind="stable")
        bq = order[:, 0]
        best_q[live, t] = bq
        best[live, t] = score[rows, bq]
        A = _gram3(G1, G2, G3, np.concatenate([prev, bq[:, None]], axis=1), n1, n2)
        _, best_piv2[live, t] = _cholesky_rows(A)
        best_Att[live, t] = A[:, t, t]
        go = nnz[live] > t
        idx = live[go]
        if idx.size == 0:
            continue
        sel = support[idx, :t + 1]
        pick[idx, t] = score[rows[go], sel[:, t]]
        A = _gram3(G1, G2, G3, sel, n1, n2)
        Lc, pick_piv2[idx, t] = _cholesky_rows(A)
        pick_Att[idx, t] = A[:, t, t]
        x = _cholesky_solve(Lc, np.take_along_axis(C0[idx], sel, axis=1))
        coef[idx, :t + 1] = x
        R[idx] = Y[idx] - reconstruct3(D1, D2, D3, sel, x)
    res_energy = energy[np.arange(N), np.minimum(nnz, s)]
    return ReplayResult(energy=energy, best=best, best_q=best_q, best_piv2=best_piv2,
                        best_Att=best_Att, pick=pick, pick_piv2=pick_piv2, pick_Att=pick_Att,
                        coef=coef, res_energy=res_energy)


class Update3Result:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def update_mode(Y, Ds, support, coef, k: int) -> Update3Result:
    """Remark 3 for mode k (0, 1, 2): P = sum X_(k) T^T T X_(k)^T with T the
    Kronecker product of the other dictionaries in mode order, B = sum
    Y_(k) T X_(k)^T; D_k* = B P^{-1} on the used atoms; normalise; rescale
    the coefficients of every pick by the norm of its mode-k atom."""
    Y = np.asarray(Y, dtype=np.float64)
    ns = [D.shape[1] for D in Ds]
    others = [m for m in range(3) if m != k]
    T = np.kron(Ds[others[1]], Ds[others[0]])          # the later mode is the outer factor
    X = densify3(support, coef, *ns)
    P = np.zeros((ns[k], ns[k]))
    B = np.zeros((Ds[k].shape[0], ns[k]))
    for idx in range(len(Y)):
        Xk = unfold(X[idx], k)
        Yk = unfold(Y[idx], k)
        XT = Xk @ T.T
        P += XT @ XT.T
        B += Yk @ XT.T
    Dstar, D, norms, used = _solve_normal(P, B, np.asarray(Ds[k], dtype=np.float64))
    valid = support >= 0
    q = np.where(valid, support, 0)
    atom = [q % ns[0], (q // ns[0]) % ns[1], q // (ns[0] * ns[1])][k]
    new_coef = np.where(valid, coef * norms[atom], 0.0)
    newDs = list(Ds)
    newDs[k] = D
    return Update3Result(D=D, coef=new_coef, P=P, B=B, used=used, norms=norms,
                         obj_before=objective3(Y, *Ds, support, coef),
                         obj_after=objective3(Y, *newDs, support, new_coef))


class Iter3Result:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def iterate3(Y, D1, D2, D3, s: int) -> Iter3Result:
    """Code, D1 update, code, D2 update, code, D3 update; the RMSE right after
    each update (with the codes of the preceding coding pass, rescaled)."""
    Y = np.asarray(Y, dtype=np.float64)
    scale = Y.size
    Ds = [np.asarray(D, dtype=np.float64) for D in (D1, D2, D3)]
    rmse, codes = [], []
    for k in range(3):
        code = omp3d(Y, *Ds, s)
        upd = update_mode(Y, Ds, code.support, code.coef, k)
        Ds[k] = upd.D
        rmse.append(float(np.sqrt(upd.obj_after / scale)))
        codes.append((code, upd))
    return Iter3Result(D=Ds, rmse=rmse, support=codes[-1][0].support, coef=codes[-1][1].coef,
                       nnz=codes[-1][0].nnz, passes=codes)
