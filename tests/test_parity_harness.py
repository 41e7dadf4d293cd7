"""The parity harness itself, on the CPU: codes planted from the oracle's own
results (with deliberate ties, threshold decisions and mistakes) must be
classified as the module docstring of tests/parity.py says."""
import numpy as np
import pytest

import oracle
from paper_2007_03800_gb300 import synth
from parity import check_codes


def problem(N=300, seed=11):
    Y, _, _, _, _ = synth.kron_model(N, 8, 8, 16, 16, 4, 20.0, seed=seed)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    return Y, D1, D2


def test_oracle_codes_are_exact():
    Y, D1, D2 = problem()
    ref = oracle.omp2d(Y, D1, D2, 4)
    rep = check_codes(Y, D1, D2, 4, ref.support, ref.nnz, ref.coef, ref.res_energy, ref=ref)
    assert rep.exact == rep.n and rep.bad == 0 and rep.coef_err < 1e-12
    rep.assert_ok()


def test_wrong_pick_is_bad():
    """A second-best pick far outside the tie window is a mismatch."""
    Y, D1, D2 = problem()
    ref = oracle.omp2d(Y, D1, D2, 4)
    k = int(np.argmax(ref.top_val[:, 1, 1] < 0.9 * ref.top_val[:, 1, 0]))
    sup = ref.support.copy()
    sup[k, 1] = ref.top_q[k, 1, 1]
    sup[k, 2:] = -1
    nnz = ref.nnz.copy()
    nnz[k] = 2
    rep = check_codes(Y, D1, D2, 4, sup, nnz, ref=ref)
    assert rep.bad == 1 and rep.bad_examples[0][0] == k
    with pytest.raises(AssertionError):
        rep.assert_ok()


def test_exact_tie_taken_the_other_way_is_a_checked_tie():
    """Duplicated atom: pairs (3, j) and (5, j) score exactly the same.  Codes
    that take the larger q are a tie; their coefficients are still checked
    against the oracle's fit on that support, so a wrong coefficient fails."""
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    D1[:, 5] = D1[:, 3]
    rng = np.random.default_rng(9)
    N = 40
    j = rng.integers(0, 16, N)
    Y = np.einsum("a,kb->kab", D1[:, 3], D2[:, j].T) * rng.uniform(1.0, 2.0, (N, 1, 1))
    Y += 1e-3 * rng.standard_normal(Y.shape)
    ref = oracle.omp2d(Y, D1, D2, 4)
    assert np.all(ref.support[:, 0] == 3 + 16 * j)
    sup = ref.support.copy()
    sup[0, 0] = 5 + 16 * j[0]            # the other copy: same score, same fit
    rep = check_codes(Y, D1, D2, 4, sup, ref.nnz, ref.coef, ref.res_energy, ref=ref)
    assert rep.ties == 1 and rep.bad == 0 and rep.tie_rows[0]
    assert rep.coef_err < 1e-10
    coef = ref.coef.copy()
    coef[0, 0] *= 1.001
    rep2 = check_codes(Y, D1, D2, 4, sup, ref.nnz, coef, ref.res_energy, ref=ref)
    assert rep2.coef_err > 1e-4
    with pytest.raises(AssertionError):
        rep2.assert_ok()


def test_tie_bound_is_enforced():
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    D1[:, 5] = D1[:, 3]
    rng = np.random.default_rng(9)
    N = 40
    j = rng.integers(0, 16, N)
    Y = np.einsum("a,kb->kab", D1[:, 3], D2[:, j].T) * rng.uniform(1.0, 2.0, (N, 1, 1))
    Y += 1e-3 * rng.standard_normal(Y.shape)
    ref = oracle.omp2d(Y, D1, D2, 4)
    sup = ref.support.copy()
    sup[:10, 0] = 5 + 16 * j[:10]
    rep = check_codes(Y, D1, D2, 4, sup, ref.nnz, ref=ref)
    assert rep.ties == 10 and rep.bad == 0
    with pytest.raises(AssertionError):
        rep.assert_ok()           # 10 ties > max(2, 2e-3 * 40)


def test_error_target_window():
    """Error-driven mode: continuing past the target is allowed only when the
    residual energy sits within EPS_WIN ||Y||^2 of eps^2."""
    Y, D1, D2 = problem(N=50, seed=3)
    free = oracle.omp2d(Y, D1, D2, 4)
    k = 7
    e_t = oracle.omp2d_replay(Y[k:k + 1], D1, D2, free.support[k:k + 1], free.nnz[k:k + 1], 4).energy[0]
    # eps just above ||R|| after two picks: the oracle stops at two, codes with three are a threshold case
    eps = float(np.sqrt(e_t[2] * (1 + 1e-8)))
    ref = oracle.omp2d(Y, D1, D2, 4, eps=eps)
    assert ref.nnz[k] == 2
    sup = ref.support.copy()
    nnz = ref.nnz.copy()
    sup[k, 2] = free.support[k, 2]
    nnz[k] = 3
    rep = check_codes(Y, D1, D2, 4, sup, nnz, eps=eps, ref=ref)
    assert rep.threshold == 1 and rep.bad == 0
    # the same extra pick with eps far above ||R||: a mismatch
    eps_far = float(np.sqrt(e_t[2] * 1.5))
    ref_far = oracle.omp2d(Y, D1, D2, 4, eps=eps_far)
    sup2 = ref_far.support.copy()
    nnz2 = ref_far.nnz.copy()
    assert nnz2[k] <= 2
    sup2[k, :3] = free.support[k, :3]
    nnz2[k] = 3
    rep2 = check_codes(Y, D1, D2, 4, sup2, nnz2, eps=eps_far, ref=ref_far)
    assert rep2.bad >= 1 and any(b[0] == k for b in rep2.bad_examples)


def test_unexplained_early_stop_is_bad():
    Y, D1, D2 = problem()
    ref = oracle.omp2d(Y, D1, D2, 4)
    sup = ref.support.copy()
    nnz = ref.nnz.copy()
    sup[3, 2:] = -1
    nnz[3] = 2
    rep = check_codes(Y, D1, D2, 4, sup, nnz, ref=ref)
    assert rep.bad == 1 and rep.bad_examples[0][1] == "stopped early"
