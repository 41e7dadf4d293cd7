"""Comparison helpers between the CUDA path and the FP64 oracle.

Codes.  A signal whose GPU pick sequence equals the oracle's (and stops at
the same step) is "exact".  Any other signal is replayed by the oracle along
the GPU's own picks (oracle.omp2d_replay) and every step of that path is
judged by the rule of Sec. III step 1:

  * a pick must score within TIE_REL of the best unselected score at its
    step (a "tie" when it is not the rule's own choice there);
  * a pick the oracle would refuse (Cholesky pivot^2 <= PIVOT_REL A_tt) or,
    in error-driven mode, a pick made with ||R||^2 <= eps^2, is allowed only
    inside a window around that threshold ("threshold": pivot^2 within a
    factor PIV_WIN of it; | ||R||^2 - eps^2 | <= EPS_WIN ||Y||^2);
  * a stop before s picks must be explained by the best score being zero,
    a degenerate pivot of the best pair, or ||R||^2 <= eps^2, each within the
    same windows;

anything else is "bad".  The coefficients and residual energy of every
signal that is not bad are then compared with the oracle's least-squares fit
on the GPU's own support (the oracle's omp2d result for exact signals, the
replay for the others), so signals with a tie are checked too.  Ties and
threshold decisions together are bounded per call (assert_ok).
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2007_03800_gb300 import sdl

TIE_REL = 1e-6       # relative score window of an argmax tie
EPS_WIN = 1e-5       # | ||R||^2 - eps^2 | window at the error-driven stop, relative to ||Y||^2
PIV_WIN = 10.0       # factor around PIVOT_REL inside which a degenerate-pick decision may differ
ZERO_REL = 1e-6      # a best score below ZERO_REL ||Y|| may stop a signal (FP32 exact zero)
COEF_RTOL = 1e-4     # per-signal ||x_gpu - x_ref|| / ||x_ref||
ENERGY_RTOL = 1e-3   # |E_gpu - E_ref| <= ENERGY_RTOL E_ref + ENERGY_ABS ||Y||^2, where
ENERGY_ABS = 2e-6    # the FP32 energy identity ||Y||^2 - sum_t y_t^2 rounds at most
                     # s + 1 <= 33 times at magnitudes <= ||Y||^2 (33 x 2^-24 < 2e-6)
DICT_RTOL = 1e-4     # max |D_gpu - D_ref| (unit-norm columns)
RMSE_RTOL = 1e-4
MAX_TIE_FRAC = 2e-3  # ties + threshold decisions <= max(2, MAX_TIE_FRAC n)


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


class CodeReport:
    """Outcome of check_codes.  exact_rows / ok_rows: boolean masks (exact,
    and not bad); ref_coef / ref_energy: the oracle's coefficients and
    residual energies along every signal's GPU path (valid on ok_rows)."""

    def __init__(self, n, exact_rows, tie_rows, thr_rows, bad, ref_coef, ref_energy,
                 coef_err, energy_err):
        self.n = n
        self.exact_rows, self.tie_rows, self.thr_rows = exact_rows, tie_rows, thr_rows
        self.exact, self.ties, self.threshold = int(exact_rows.sum()), int(tie_rows.sum()), int(thr_rows.sum())
        self.bad_examples = bad
        self.bad = len(bad)
        self.ok_rows = exact_rows | tie_rows | thr_rows
        self.ref_coef, self.ref_energy = ref_coef, ref_energy
        self.coef_err, self.energy_err = coef_err, energy_err

    def __repr__(self):
        return (f"CodeReport(n={self.n}, exact={self.exact}, ties={self.ties}, "
                f"threshold={self.threshold}, bad={self.bad}, coef_err={self.coef_err:.2e}, "
                f"energy_err={self.energy_err:.2e}, examples={self.bad_examples[:3]})")

    def assert_ok(self, max_tie_frac=MAX_TIE_FRAC, coef_rtol=COEF_RTOL, energy_rtol=ENERGY_RTOL):
        print(f"parity: n={self.n} exact={self.exact} ties={self.ties} threshold={self.threshold} "
              f"coef_err={self.coef_err:.2e} energy_err={self.energy_err:.2e}")
        assert self.bad == 0, self
        assert self.ties + self.threshold <= max(2, max_tie_frac * self.n), self
        assert self.coef_err < coef_rtol, self
        assert self.energy_err < energy_rtol, self


def _judge(rp, sup, nnz, s, eps2, ynorm2, tie_rel):
    """Classify the replayed signals: 0 = valid path without special steps,
    1 = a tie was taken, 2 = a threshold decision differed; returns (cls,
    reason) with cls = -1 and a reason for a bad signal."""
    m = sup.shape[0]
    cls = np.zeros(m, dtype=np.int64)
    reason = [None] * m
    thr_piv = oracle.PIVOT_REL
    for k in range(m):
        tie = thr = False
        why = None
        for t in range(int(nnz[k])):
            best, pick = rp.best[k, t], rp.pick[k, t]
            if not (pick >= 0 and pick >= (1.0 - tie_rel) * best):
                why = ("pick below the tie window", t, float(pick), float(best))
                break
            if sup[k, t] != rp.best_q[k, t]:
                tie = True
            piv, att = rp.pick_piv2[k, t], rp.pick_Att[k, t]
            if piv <= thr_piv * att:
                if piv <= thr_piv * att / PIV_WIN:
                    why = ("degenerate pick accepted", t, float(piv / att))
                    break
                thr = True
            if eps2 is not None and rp.energy[k, t] <= eps2:
                if eps2 - rp.energy[k, t] > EPS_WIN * ynorm2[k]:
                    why = ("pick below the error target", t, float(rp.energy[k, t]), eps2)
                    break
                thr = True
        t = int(nnz[k])
        if why is None and t < s:
            # the GPU stopped at step t: some stop rule must (nearly) hold there
            e_t, best = rp.energy[k, t], rp.best[k, t]
            piv, att = rp.best_piv2[k, t], rp.best_Att[k, t]
            if eps2 is not None and e_t <= eps2:
                pass
            elif eps2 is not None and e_t - eps2 <= EPS_WIN * ynorm2[k]:
                thr = True
            elif best == 0.0:
                pass
            elif best <= ZERO_REL * np.sqrt(ynorm2[k]):
                thr = True
            elif piv <= thr_piv * att:
                pass
            elif piv <= PIV_WIN * thr_piv * att:
                thr = True
            else:
                why = ("stopped early", t, float(e_t), float(best), float(piv / att))
        if why is not None:
            cls[k], reason[k] = -1, why
        else:
            cls[k] = 1 if tie else (2 if thr else 0)
    return cls, reason


def check_codes(Y, D1, D2, s, sup, nnz, coef=None, energy=None, eps=None, ref=None,
                tie_rel=TIE_REL, replay=None):
    """Judge GPU codes (support, nnz and optionally coef, res_energy) of the
    signals Y against the oracle (see the module docstring).  replay: the
    oracle's forced-support replay (default the two-mode one, with D1, D2);
    three-mode codes pass their own with ref."""
    Y = np.asarray(Y, dtype=np.float64)
    sup = np.asarray(sup).astype(np.int64)
    nnz = np.asarray(nnz).astype(np.int64)
    if ref is None:
        ref = oracle.omp2d(Y, D1, D2, s, eps=eps)
    n = sup.shape[0]
    ynorm2 = np.sum(Y * Y, axis=tuple(range(1, Y.ndim)))
    eps2 = None if eps is None else float(eps) ** 2
    exact = np.all(sup == ref.support, axis=1) & (nnz == ref.nnz)
    ref_coef = np.where(exact[:, None], ref.coef, 0.0)
    ref_energy = np.where(exact, ref.res_energy, np.nan)
    tie_rows = np.zeros(n, dtype=bool)
    thr_rows = np.zeros(n, dtype=bool)
    bad = []
    others = np.nonzero(~exact)[0]
    if others.size:
        rp = (replay or (lambda Yo, so, no: oracle.omp2d_replay(Yo, D1, D2, so, no, s)))(
            Y[others], sup[others], nnz[others])
        cls, reason = _judge(rp, sup[others], nnz[others], s, eps2, ynorm2[others], tie_rel)
        for r, k in enumerate(others):
            if cls[r] < 0:
                bad.append((int(k),) + tuple(reason[r]))
            elif cls[r] == 0:
                bad.append((int(k), "differs from the oracle without a tie or threshold step"))
            else:
                (tie_rows if cls[r] == 1 else thr_rows)[k] = True
                ref_coef[k] = rp.coef[r]
                ref_energy[k] = rp.res_energy[r]
    ok = exact | tie_rows | thr_rows
    coef_err = energy_err = 0.0
    if coef is not None and ok.any():
        coef_err = float(coef_rel_error(coef, ref_coef, ok).max())
    if energy is not None and ok.any():
        e = np.asarray(energy, dtype=np.float64)[ok]
        # in units of the allowed error (<= ENERGY_RTOL passes): relative for
        # large residuals, relative to ||Y||^2 for residuals near zero
        allowed = (ENERGY_RTOL * ref_energy[ok] + ENERGY_ABS * ynorm2[ok]) / ENERGY_RTOL
        diff = np.abs(e - ref_energy[ok])
        energy_err = float(np.max(np.where(allowed > 0, diff / np.where(allowed > 0, allowed, 1.0),
                                           diff)))   # zero signals: exact
    return CodeReport(n, exact, tie_rows, thr_rows, bad, ref_coef, ref_energy, coef_err, energy_err)


def check_iteration(Y, D1, D2, s, support, nnz, coef, D1_gpu, D2_gpu, rmse_gpu=None, eps=None,
                    ref=None, dict_rtol=DICT_RTOL, rmse_rtol=RMSE_RTOL, max_tie_frac=MAX_TIE_FRAC):
    """One Algorithm-1 iteration on the GPU against the oracle: D1 after the
    D1 update; the second coding pass judged by check_codes with the oracle's
    new D1; then the D2 update replayed by the oracle on the GPU's own
    supports (with the oracle's coefficients along them), against which the
    GPU's D2, its rescaled coefficients and both RMSEs are compared."""
    Y = np.asarray(Y, dtype=np.float64)
    if ref is None:
        ref = oracle.iterate(Y, D1, D2, s, eps=eps)
    N, p1, p2 = Y.shape
    rep = check_codes(Y, ref.upd_a.D, D2, s, support, nnz, eps=eps, ref=ref.omp_b)
    rep.assert_ok(max_tie_frac=max_tie_frac)
    sup = np.where(rep.ok_rows[:, None], np.asarray(support).astype(np.int64), -1)
    upd = oracle.update_D2(Y, ref.upd_a.D, D2, sup, rep.ref_coef)
    d1 = np.abs(np.asarray(D1_gpu, dtype=np.float64) - ref.D1).max()
    d2 = np.abs(np.asarray(D2_gpu, dtype=np.float64) - upd.D).max()
    assert d1 < dict_rtol, ("D1", d1)
    assert d2 < dict_rtol, ("D2", d2)
    cerr = coef_rel_error(coef, upd.coef, rep.ok_rows).max(initial=0.0)
    assert cerr < COEF_RTOL, ("coef after the D2 rescale", cerr)
    if rmse_gpu is not None:
        r = np.asarray(rmse_gpu, dtype=np.float64)
        want1 = ref.rmse_after_D1
        want2 = float(np.sqrt(upd.obj_after / (p1 * p2 * N)))
        assert abs(r[0] - want1) / want1 < rmse_rtol, ("rmse after D1", r[0], want1)
        assert abs(r[1] - want2) / want2 < rmse_rtol, ("rmse after D2", r[1], want2)
    return rep, upd


def coef_rel_error(gpu_coef, ref_coef, rows):
    g = np.asarray(gpu_coef, dtype=np.float64)[rows]
    r = np.asarray(ref_coef)[rows]
    num = np.linalg.norm(g - r, axis=1)
    den = np.maximum(np.linalg.norm(r, axis=1), 1e-30)
    return num / den
