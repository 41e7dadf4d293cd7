"""FP64 reference of the orthonormal variant of Algorithm 1 (Remark 1 of Rusu &
Irofti, arXiv 2007.03800): square orthonormal dictionaries, hard-thresholded
codes and orthogonal-Procrustes dictionary updates.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What each routine follows:
  threshold_code : X_k = T_s(D1^T Y_k D2), the s largest |entries| kept
                   (Remark 1); exact ties go to the smallest q = i + n1*j
  procrustes_D1  : with X fixed and D1 orthonormal, Eq. (1) equals
                   const - 2 tr(D1^T B1), B1 = sum_k Y_k D2 X_k^T; its maximiser is
                   the orthogonal polar factor D1* = U V^T of B1 = U S V^T
  procrustes_D2  : the mirror, B2 = sum_k Y_k^T D1 X_k, D2* = U2 V2^T
  iterate        : code, D1 update, code again with the new D1, D2 update
                   (the main loop of Algorithm 1 with the Procrustes updates)

Readings where the paper is garbled or silent:
  * Remark 1 prints the SVD argument as (sum Y_k^T D2 X_k)(sum X_k X_k^T); the
    dimensions only agree for square signals and the extra factor is not the
    Procrustes matrix.  Maximising tr(D1^T sum_k Y_k D2 X_k^T) over orthonormal
    D1 gives the SVD of B1 = sum_k Y_k D2 X_k^T alone (and of
    B2 = sum_k Y_k^T D1 X_k for D2), which is what is computed here.  B1 and
    B2 are the same sums as in the general update (Corollary 1, Result 1).
  * A numerically rank-deficient B has no unique Procrustes solution:
    SingularError, dictionary unchanged.  B is a sum of FP32 data, so rank
    deficiency is judged at that precision: smallest singular value <= 1e-6 of
    the largest.
"""
from __future__ import annotations

import numpy as np

from .sdl_oracle import SingularError, densify

__all__ = ["threshold_code", "procrustes_D1", "procrustes_D2", "ortho_iterate",
           "SVD_RANK_REL", "OrthoIterResult"]

SVD_RANK_REL = 1e-6
_CHUNK = 4096


def threshold_code(Y, D1, D2, s: int, eps: float | None = None):
    """T_s(D1^T Y_k D2) for every k.  Returns (support (N, s) int64 in order of
    decreasing |value|, ties by smaller q, -1 for slots whose entry is exactly
    0; coef (N, s); res_energy (N,) = ||Y_k - D1 X_k D2^T||^2 formed
    explicitly).  With eps, error-driven: before each kept entry, stop once
    the residual norm is <= eps (for orthonormal D the residual energy after
    keeping entries c_1..c_t is ||Y_k||^2 - sum c_l^2), at most s entries."""
    Y = np.asarray(Y, dtype=np.float64)
    N, p1, p2 = Y.shape
    n1, n2 = D1.shape[1], D2.shape[1]
    C = np.einsum("ai,kab,bj->kij", D1, Y, D2, optimize=True)
    flat = C.transpose(0, 2, 1).reshape(N, n1 * n2)          # entry q = i + n1*j
    # stable sort of -|C| keeps the smaller q first among equal magnitudes
    order = np.argsort(-np.abs(flat), axis=1, kind="stable")[:, :s]
    coef = np.take_along_axis(flat, order, axis=1)
    support = order.astype(np.int64)
    # exactly-zero entries are not picks (a signal then keeps fewer than s)
    zero = coef == 0.0
    if eps is not None:
        energy = np.einsum("kab,kab->k", Y, Y)
        kept_before = np.concatenate([np.zeros((N, 1)), np.cumsum(coef ** 2, axis=1)[:, :-1]], axis=1)
        zero |= (energy[:, None] - kept_before) <= eps * eps
        zero = np.logical_or.accumulate(zero, axis=1)
    support[zero] = -1
    coef[zero] = 0.0
    X = densify(support, coef, n1, n2)
    R = Y - np.einsum("ai,kij,bj->kab", D1, X, D2, optimize=True)
    return support, coef, np.einsum("kab,kab->k", R, R)


def _polar(B):
    """Orthogonal polar factor U V^T of a square B (its Procrustes maximiser)."""
    U, S, Vt = np.linalg.svd(B)
    if S[-1] <= SVD_RANK_REL * S[0]:
        raise SingularError("Procrustes matrix is numerically rank deficient")
    return U @ Vt, S


class ProcrustesResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def procrustes_D1(Y, D1, D2, support, coef) -> ProcrustesResult:
    """D1* = polar(B1), B1 = sum_k Y_k D2 X_k^T (Remark 1, D2 and X fixed)."""
    Y = np.asarray(Y, dtype=np.float64)
    n1, n2 = D1.shape[1], D2.shape[1]
    B = np.zeros((Y.shape[1], n1))
    for a in range(0, len(Y), _CHUNK):
        X = densify(support[a:a + _CHUNK], coef[a:a + _CHUNK], n1, n2)
        B += np.einsum("kab,bj,kij->ai", Y[a:a + _CHUNK], D2, X, optimize=True)
    D, S = _polar(B)
    return ProcrustesResult(D=D, B=B, sigma=S)


def procrustes_D2(Y, D1, D2, support, coef) -> ProcrustesResult:
    """D2* = polar(B2), B2 = sum_k Y_k^T D1 X_k (Remark 1, D1 and X fixed)."""
    Y = np.asarray(Y, dtype=np.float64)
    n1, n2 = D1.shape[1], D2.shape[1]
    B = np.zeros((Y.shape[2], n2))
    for a in range(0, len(Y), _CHUNK):
        X = densify(support[a:a + _CHUNK], coef[a:a + _CHUNK], n1, n2)
        B += np.einsum("kab,ai,kij->bj", Y[a:a + _CHUNK], D1, X, optimize=True)
    D, S = _polar(B)
    return ProcrustesResult(D=D, B=B, sigma=S)


class OrthoIterResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def ortho_iterate(Y, D1, D2, s: int) -> OrthoIterResult:
    """One iteration of Algorithm 1 - Orthonormal: threshold codes, D1 by
    Procrustes, codes again with the new D1, D2 by Procrustes.  The RMSEs are
    ||Y - D1 X D2^T||_F / sqrt(p1 p2 N) right after each update, with X the
    codes of the preceding coding step."""
    Y = np.asarray(Y, dtype=np.float64)
    N, p1, p2 = Y.shape
    scale = p1 * p2 * N
    sup_a, coef_a, _ = threshold_code(Y, D1, D2, s)
    upd_a = procrustes_D1(Y, D1, D2, sup_a, coef_a)
    sup_b, coef_b, res_b = threshold_code(Y, upd_a.D, D2, s)
    upd_b = procrustes_D2(Y, upd_a.D, D2, sup_b, coef_b)

    def rmse(Da, Db, sup, coef):
        X = densify(sup, coef, Da.shape[1], Db.shape[1])
        R = Y - np.einsum("ai,kij,bj->kab", Da, X, Db, optimize=True)
        return float(np.sqrt(np.sum(R * R) / scale))

    return OrthoIterResult(D1=upd_a.D, D2=upd_b.D, support=sup_b, coef=coef_b, res_energy=res_b,
                           rmse_after_D1=rmse(upd_a.D, D2, sup_a, coef_a),
                           rmse_after_D2=rmse(upd_a.D, upd_b.D, sup_b, coef_b),
                           support_a=sup_a, coef_a=coef_a, upd_a=upd_a, upd_b=upd_b)
