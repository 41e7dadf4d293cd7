"""Plain FP64 reference for separable dictionary learning (Rusu & Irofti,
"Efficient and Parallel Separable Dictionary Learning", arXiv 2007.03800).

TEST INFRASTRUCTURE ONLY: see the package docstring.  Slow and obvious on
purpose; every routine is vectorised over independent signals only (one
signal's arithmetic is never reordered or fused).

Notation follows the paper with the signal-size names p1, p2 (the paper's m):
  Y_k  p1 x p2 signal, k = 1..N           (array Y of shape (N, p1, p2))
  D1   p1 x n1 left dictionary, D2 p2 x n2 right dictionary, unit columns
  X_k  n1 x n2 sparse code with at most s nonzeros
  atom pair (i, j) <-> column q = i + n1*j of D2 (x) D1   (Sec. I, column-order vec)
Sparse codes are kept as ``support`` (N, s) int64 pair indices in pick order
(-1 = unused slot) and ``coef`` (N, s) float64 values.

What each routine follows:
  objective / rmse  : Eq. (1), the separable DL objective
  omp2d             : the 2D-OMP sparse coder of Sec. III step 1), i.e. greedy
                      pursuit over Kronecker atom pairs, equivalent to 1D OMP on
                      D2 (x) D1 (Sec. II); full least-squares re-fit per pick
  omp2d_replay      : the same pursuit forced along a given pick sequence
                      (every step's scores, pivots and residual energies on
                      that path, and the least-squares fit on its support)
  update_D1         : Corollary 1 (optimal D1, then the W1 normalisation)
  update_D2         : Result 1 (optimal D2, then the W2 normalisation)
  iterate           : one pass of the main loop of Algorithm 1 (steps 1-4)

Readings where the paper is silent or garbled:
  * Algorithm 1 prints D1 = P^{-1} R W1 and D2 = M^{-1} N W2; the dimensions
    only agree with Corollary 1 / Result 1 as D1* = (sum Y_k T_k^T) P^{-1} and
    D2* = (sum Y_k^T Z_k) M^{-1}, which is what is computed here.
  * The Gram shortcut of Sec. III prints G2 = D2 D2^T; T_k T_k^T = X_k G2 X_k^T
    needs G2 = D2^T D2 (n2 x n2).
  * 2D-OMP internals: pick argmax |<R, d1_i d2_j^T>| over pairs not yet
    selected; exact ties go to the smallest q.  Stop a signal early when the
    best score is 0, or when the new pair's Cholesky pivot satisfies
    pivot^2 <= PIVOT_REL * A_tt (a pair numerically inside the span of the
    selected ones).  In error-bounded mode stop before a pick once
    ||R||_F <= eps (Sec. IV denoising: error-driven OMP capped at s).
  * An atom that no signal uses gives a zero row/column in P (or M): the normal
    equations are solved on the used atoms only and unused atoms are kept.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

__all__ = [
    "PIVOT_REL", "grams", "reconstruct", "residual", "objective", "rmse",
    "densify", "omp2d", "omp2d_replay", "ReplayResult", "update_D1", "update_D2", "iterate",
    "OMPResult", "UpdateResult", "IterResult", "SingularError",
]

PIVOT_REL = 1e-6          # degenerate-pick threshold on pivot^2 / A_tt
_CHUNK = 4096             # signals per block (memory only; sums are plain)


class SingularError(RuntimeError):
    """The normal-equation matrix of a dictionary update is not SPD."""


# --------------------------------------------------------------------------
# Objective, Eq. (1)
# --------------------------------------------------------------------------
def grams(D1: np.ndarray, D2: np.ndarray):
    """G1 = D1^T D1 and G2 = D2^T D2 (Sec. III, G2 read as D2^T D2)."""
    return D1.T @ D1, D2.T @ D2


def reconstruct(D1, D2, support, coef):
    """D1 X_k D2^T for every k, summing x_l d1_{i_l} d2_{j_l}^T over the support."""
    n1 = D1.shape[1]
    valid = support >= 0
    q = np.where(valid, support, 0)
    i, j = q % n1, q // n1
    x = np.where(valid, coef, 0.0)
    return np.einsum("kl,akl,bkl->kab", x, D1[:, i], D2[:, j], optimize=True)


def residual(Y, D1, D2, support, coef):
    """R_k = Y_k - D1 X_k D2^T."""
    return Y - reconstruct(D1, D2, support, coef)


def objective(Y, D1, D2, support, coef) -> float:
    """sum_k ||Y_k - D1 X_k D2^T||_F^2, the objective of Eq. (1)."""
    total = 0.0
    for a in range(0, Y.shape[0], _CHUNK):
        R = residual(Y[a:a + _CHUNK], D1, D2, support[a:a + _CHUNK], coef[a:a + _CHUNK])
        total += float(np.sum(R * R))
    return total


def rmse(Y, D1, D2, support, coef) -> float:
    """||Y - D1 X D2^T||_F / sqrt(p1 p2 N) over the whole set."""
    N, p1, p2 = Y.shape
    return float(np.sqrt(objective(Y, D1, D2, support, coef) / (p1 * p2 * N)))


def densify(support, coef, n1: int, n2: int) -> np.ndarray:
    """Dense X of shape (N, n1, n2) from (support, coef)."""
    N = support.shape[0]
    X = np.zeros((N, n1 * n2))
    valid = support >= 0
    rows = np.repeat(np.arange(N)[:, None], support.shape[1], axis=1)
    np.add.at(X, (rows[valid], support[valid]), coef[valid])
    return X.reshape(N, n2, n1).transpose(0, 2, 1)


# --------------------------------------------------------------------------
# 2D-OMP (Sec. III step 1; equivalent to 1D OMP on D2 (x) D1, Sec. II)
# --------------------------------------------------------------------------
class OMPResult:
    """support (N, s) int64, coef (N, s), nnz (N,), res_energy (N,) = ||R_k||^2,
    and for tie analysis, per pick step: top_q / top_val (N, s, K) the K best
    unselected pairs by |correlation| (descending, ties by smaller q)."""

    def __init__(self, support, coef, nnz, res_energy, top_q, top_val):
        self.support, self.coef, self.nnz = support, coef, nnz
        self.res_energy, self.top_q, self.top_val = res_energy, top_q, top_val


def _cholesky_rows(A):
    """Lower Cholesky factor of a batch of small SPD matrices, by the textbook
    column recurrence, plus the pivot^2 of the last column (for the
    degenerate-pick rule).  A: (m, t, t)."""
    m, t, _ = A.shape
    L = np.zeros_like(A)
    piv2 = np.zeros(m)
    for c in range(t):
        d = A[:, c, c] - np.sum(L[:, c, :c] ** 2, axis=1)
        piv2 = d
        Lcc = np.sqrt(np.maximum(d, np.finfo(float).tiny))
        L[:, c, c] = Lcc
        for r in range(c + 1, t):
            L[:, r, c] = (A[:, r, c] - np.sum(L[:, r, :c] * L[:, c, :c], axis=1)) / Lcc
    return L, piv2


def _cholesky_solve(L, b):
    """Solve L L^T x = b for a batch (forward then back substitution)."""
    m, t, _ = L.shape
    z = np.zeros((m, t))
    for r in range(t):
        z[:, r] = (b[:, r] - np.sum(L[:, r, :r] * z[:, :r], axis=1)) / L[:, r, r]
    x = np.zeros((m, t))
    for r in range(t - 1, -1, -1):
        x[:, r] = (z[:, r] - np.sum(L[:, r + 1:, r] * x[:, r + 1:], axis=1)) / L[:, r, r]
    return x


def omp2d(Y, D1, D2, s: int, eps: float | None = None, top_k: int = 4) -> OMPResult:
    """2D-OMP of every signal in Y with the pair dictionary (D1, D2).

    Per signal, starting from R = Y and an empty support, for t = 1..s:
      (error mode) stop if ||R||_F <= eps;
      C = D1^T R D2 (correlation of R with every atom pair d1_i d2_j^T);
      pick q = argmax |C_q| over unselected pairs (ties -> smallest q);
      stop if that maximum is 0;
      re-fit all coefficients: minimise ||Y - sum_l x_l d1_{i_l} d2_{j_l}^T||_F
        through a fresh Cholesky of A[l,l'] = G1[i_l,i_l'] G2[j_l,j_l'] with
        right-hand side b_l = (D1^T Y D2)[i_l, j_l]; stop instead of adding the
        pair if its pivot is degenerate (pivot^2 <= PIVOT_REL * A_tt);
      R = Y - D1 X D2^T, formed explicitly.
    """
    Y = np.asarray(Y, dtype=np.float64)
    D1 = np.asarray(D1, dtype=np.float64)
    D2 = np.asarray(D2, dtype=np.float64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    nq = n1 * n2
    if not 1 <= s <= min(p1 * p2, nq):
        raise ValueError("need 1 <= s <= min(p1*p2, n1*n2)")
    G1, G2 = grams(D1, D2)
    C0 = np.einsum("ai,kab,bj->kij", D1, Y, D2, optimize=True)
    support = np.full((N, s), -1, dtype=np.int64)
    coef = np.zeros((N, s))
    nnz = np.zeros(N, dtype=np.int64)
    K = min(top_k, nq)
    top_q = np.full((N, s, K), -1, dtype=np.int64)
    top_val = np.full((N, s, K), np.nan)
    R = Y.copy()
    active = np.ones(N, dtype=bool)
    for t in range(s):
        if eps is not None:
            active &= np.sqrt(np.sum(R * R, axis=(1, 2))) > eps
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        C = np.einsum("ai,kab,bj->kij", D1, R[idx], D2, optimize=True)
        score = np.abs(C).transpose(0, 2, 1).reshape(idx.size, nq)   # column q = i + n1*j
        rows = np.arange(idx.size)
        for l in range(t):
            score[rows, support[idx, l]] = -1.0                       # mask selected pairs
        order = np.lexsort((np.broadcast_to(np.arange(nq), score.shape), -score), axis=1)[:, :K]
        top_q[idx, t] = order
        top_val[idx, t] = np.take_along_axis(score, order, axis=1)
        q = order[:, 0]                                              # smallest q among equal maxima
        best = score[rows, q]
        sup = np.concatenate([support[idx, :t], q[:, None]], axis=1)
        ii, jj = sup % n1, sup // n1
        A = G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]]
        b = C0[idx[:, None], ii, jj]
        L, piv2 = _cholesky_rows(A)
        accept = (best > 0) & (piv2 > PIVOT_REL * A[:, t, t])
        x = _cholesky_solve(L, b)
        acc = idx[accept]
        support[acc, t] = q[accept]
        coef[acc, :t + 1] = x[accept]
        nnz[acc] = t + 1
        R[acc] = Y[acc] - reconstruct(D1, D2, support[acc, :t + 1], coef[acc, :t + 1])
        active[idx[~accept]] = False
    res_energy = np.sum(R * R, axis=(1, 2))
    return OMPResult(support, coef, nnz, res_energy, top_q, top_val)


class ReplayResult:
    """Quantities of 2D-OMP along a forced pick sequence, per signal k and
    step t (t picks already made):
      energy (N, s+1)     ||R_k||^2 after t picks (R = Y - D1 X D2^T, explicit)
      best (N, s)         max |C_q| over unselected pairs at step t (NaN once
                          the sequence has ended before step t)
      best_q (N, s)       the pair the greedy rule would take there (ties ->
                          smallest q), -1 where best is NaN
      best_piv2 (N, s)    pivot^2 of best_q against the selected pairs, and
      best_Att (N, s)     its A_tt = G1[i,i] G2[j,j]
      pick (N, s)         |C_q| of the given pick at step t (-1 if that pair
                          was already selected; NaN past the sequence)
      pick_piv2, pick_Att (N, s)  the same two for the given pick
      coef (N, s)         least-squares coefficients on the whole given support
      res_energy (N,)     ||R_k||^2 after the whole sequence"""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _pivot2(G1, G2, sup_prev, q, n1):
    """pivot^2 of pair q against the selected pairs sup_prev (rows of the
    fresh Cholesky of A over sup_prev + [q]) and A_qq = G1[i,i] G2[j,j]."""
    sup = np.concatenate([sup_prev, q[:, None]], axis=1)
    ii, jj = sup % n1, sup // n1
    A = G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]]
    _, piv2 = _cholesky_rows(A)
    t = sup.shape[1] - 1
    return piv2, A[:, t, t]


def omp2d_replay(Y, D1, D2, support, nnz, s: int) -> ReplayResult:
    """2D-OMP (Sec. III step 1, 1D OMP on D2 (x) D1 by Sec. II) forced to take
    the picks support[k, :nnz[k]] in that order instead of its own argmax.

    At each step t of signal k (t = 0..nnz[k], and t < s) the residual of the
    previous least-squares fit gives the correlations C = D1^T R D2; recorded
    are the greedy rule's choice there (max |C_q| over unselected pairs, ties
    to the smallest q, with its Cholesky pivot) and, for t < nnz[k], the score
    and pivot of the forced pick, after which all coefficients are re-fitted
    on the forced support exactly as omp2d does (fresh Cholesky of A with
    b_l = (D1^T Y D2)[i_l, j_l]) and R is formed explicitly.  Used to judge a
    pick sequence that left the oracle's own path (at an argmax tie, or at
    the stop threshold): every step of it can be checked against the rule,
    and its coefficients and residual energies against this fit."""
    Y = np.asarray(Y, dtype=np.float64)
    D1 = np.asarray(D1, dtype=np.float64)
    D2 = np.asarray(D2, dtype=np.float64)
    support = np.asarray(support, dtype=np.int64)
    nnz = np.asarray(nnz, dtype=np.int64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    nq = n1 * n2
    G1, G2 = grams(D1, D2)
    C0 = np.einsum("ai,kab,bj->kij", D1, Y, D2, optimize=True)
    nan = lambda: np.full((N, s), np.nan)
    energy = np.full((N, s + 1), np.nan)
    best, best_piv2, best_Att = nan(), nan(), nan()
    pick, pick_piv2, pick_Att = nan(), nan(), nan()
    best_q = np.full((N, s), -1, dtype=np.int64)
    coef = np.zeros((N, s))
    R = Y.copy()
    for t in range(s + 1):
        live = np.nonzero(nnz >= t)[0]                 # signals that reach step t
        energy[live, t] = np.sum(R[live] ** 2, axis=(1, 2))
        if t == s or live.size == 0:
            continue
        C = np.einsum("ai,kab,bj->kij", D1, R[live], D2, optimize=True)
        score = np.abs(C).transpose(0, 2, 1).reshape(live.size, nq)   # column q = i + n1*j
        rows = np.arange(live.size)
        prev = support[live, :t]
        for l in range(t):
            score[rows, prev[:, l]] = -1.0                             # mask selected pairs
        order = np.lexsort((np.broadcast_to(np.arange(nq), score.shape), -score), axis=1)
        bq = order[:, 0]
        best_q[live, t] = bq
        best[live, t] = score[rows, bq]
        best_piv2[live, t], best_Att[live, t] = _pivot2(G1, G2, prev, bq, n1)
        go = nnz[live] > t                                           # a forced pick at step t
        idx = live[go]
        if idx.size == 0:
            continue
        q = support[idx, t]
        pick[idx, t] = score[rows[go], q]
        pick_piv2[idx, t], pick_Att[idx, t] = _pivot2(G1, G2, support[idx, :t], q, n1)
        sup = support[idx, :t + 1]
        ii, jj = sup % n1, sup // n1
        A = G1[ii[:, :, None], ii[:, None, :]] * G2[jj[:, :, None], jj[:, None, :]]
        L, _ = _cholesky_rows(A)
        x = _cholesky_solve(L, C0[idx[:, None], ii, jj])
        coef[idx, :t + 1] = x
        R[idx] = Y[idx] - reconstruct(D1, D2, sup, x)
    res_energy = energy[np.arange(N), np.minimum(nnz, s)]
    return ReplayResult(energy=energy, best=best, best_q=best_q, best_piv2=best_piv2,
                        best_Att=best_Att, pick=pick, pick_piv2=pick_piv2, pick_Att=pick_Att,
                        coef=coef, res_energy=res_energy)


# --------------------------------------------------------------------------
# TMOD dictionary updates (Corollary 1, Result 1)
# --------------------------------------------------------------------------
class UpdateResult:
    """D (new, unit columns), coef (rescaled by W^{-1}), P (the n x n normal
    matrix), B (the p x n right-hand side), Dstar (before normalisation),
    norms (column norms of Dstar; 1 for unused atoms), used (bool mask),
    obj_before / obj_after (Eq. (1) at the old and the new dictionary)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _solve_normal(P, B, D_old):
    """D* = B P^{-1} on the used atoms (diag(P) > 0); unused atoms keep their
    old column.  Cholesky of the used block (SPD when the codes have full rank)."""
    used = np.diag(P) > 0
    Dstar = D_old.copy()
    if used.any():
        Pu = P[np.ix_(used, used)]
        try:
            cf = scipy.linalg.cho_factor(Pu, lower=True)
        except np.linalg.LinAlgError as e:
            raise SingularError(str(e)) from None
        Dstar[:, used] = scipy.linalg.cho_solve(cf, B[:, used].T).T
    norms = np.ones(P.shape[0])
    norms[used] = np.linalg.norm(Dstar[:, used], axis=0)
    D = Dstar.copy()
    D[:, used] = Dstar[:, used] / norms[used]
    return Dstar, D, norms, used


def update_D1(Y, D1, D2, support, coef) -> UpdateResult:
    """Corollary 1 with X fixed: T_k = X_k D2^T, P = sum_k T_k T_k^T,
    B1 = sum_k Y_k T_k^T, D1* = B1 P^{-1}; W1 = diag(1/||d1*_i||);
    D1 <- D1* W1 and X_k <- W1^{-1} X_k (row i of every X_k times ||d1*_i||)."""
    Y = np.asarray(Y, dtype=np.float64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    P = np.zeros((n1, n1))
    B = np.zeros((p1, n1))
    for a in range(0, N, _CHUNK):
        X = densify(support[a:a + _CHUNK], coef[a:a + _CHUNK], n1, n2)
        T = X @ D2.T                                   # (k, n1, p2)
        P += np.einsum("kiq,kjq->ij", T, T)
        B += np.einsum("kaq,kiq->ai", Y[a:a + _CHUNK], T)
    Dstar, D, norms, used = _solve_normal(P, B, np.asarray(D1, dtype=np.float64))
    valid = support >= 0
    i = np.where(valid, support, 0) % n1
    new_coef = np.where(valid, coef * norms[i], 0.0)
    return UpdateResult(D=D, coef=new_coef, P=P, B=B, Dstar=Dstar, norms=norms, used=used,
                        obj_before=objective(Y, D1, D2, support, coef),
                        obj_after=objective(Y, D, D2, support, new_coef))


def update_D2(Y, D1, D2, support, coef) -> UpdateResult:
    """Result 1 with X fixed: Z_k = D1 X_k, M = sum_k Z_k^T Z_k,
    B2 = sum_k Y_k^T Z_k, D2* = B2 M^{-1} (the transpose of the printed
    (D2*)^T = M^{-1} sum Z^T Y); W2 = diag(1/||d2*_j||); D2 <- D2* W2 and
    X_k <- X_k W2^{-1} (column j of every X_k times ||d2*_j||)."""
    Y = np.asarray(Y, dtype=np.float64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    M = np.zeros((n2, n2))
    B = np.zeros((p2, n2))
    for a in range(0, N, _CHUNK):
        X = densify(support[a:a + _CHUNK], coef[a:a + _CHUNK], n1, n2)
        Z = D1 @ X                                     # (k, p1, n2)
        M += np.einsum("kai,kaj->ij", Z, Z)
        B += np.einsum("kab,kaj->bj", Y[a:a + _CHUNK], Z)
    Dstar, D, norms, used = _solve_normal(M, B, np.asarray(D2, dtype=np.float64))
    valid = support >= 0
    j = np.where(valid, support, 0) // n1
    new_coef = np.where(valid, coef * norms[j], 0.0)
    return UpdateResult(D=D, coef=new_coef, P=M, B=B, Dstar=Dstar, norms=norms, used=used,
                        obj_before=objective(Y, D1, D2, support, coef),
                        obj_after=objective(Y, D1, D, support, new_coef))


# --------------------------------------------------------------------------
# One iteration of Algorithm 1
# --------------------------------------------------------------------------
class IterResult:
    """D1, D2 after the iteration; support / coef / nnz of the second coding
    pass rescaled by W2^{-1}; rmse_after_D1 / rmse_after_D2 (RMSE right after
    each dictionary update); omp_a / omp_b the two coding passes; upd_a / upd_b
    the two updates."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def iterate(Y, D1, D2, s: int, eps: float | None = None, top_k: int = 4) -> IterResult:
    """Algorithm 1 main-loop body: 1) code all signals, 2) D1 update
    (Corollary 1), 3) code again with the new D1, 4) D2 update (Result 1)."""
    Y = np.asarray(Y, dtype=np.float64)
    N, p1, p2 = Y.shape
    scale = p1 * p2 * N
    omp_a = omp2d(Y, D1, D2, s, eps, top_k)
    upd_a = update_D1(Y, D1, D2, omp_a.support, omp_a.coef)
    omp_b = omp2d(Y, upd_a.D, D2, s, eps, top_k)
    upd_b = update_D2(Y, upd_a.D, D2, omp_b.support, omp_b.coef)
    return IterResult(D1=upd_a.D, D2=upd_b.D, support=omp_b.support, coef=upd_b.coef,
                      nnz=omp_b.nnz,
                      rmse_after_D1=float(np.sqrt(upd_a.obj_after / scale)),
                      rmse_after_D2=float(np.sqrt(upd_b.obj_after / scale)),
                      omp_a=omp_a, omp_b=omp_b, upd_a=upd_a, upd_b=upd_b)
