"""Planted mistakes in the oracle (on the CPU): each mutant below breaks one
step of the method the way a plausible bug would, and the pins of
tests/test_oracle_pins.py and the hand-worked examples of tests/golden/ must
catch every one of them.  The mutants are
installed with monkeypatch and vanish after each test."""
import numpy as np
import pytest

import oracle
from oracle import sdl_oracle as so
import test_golden as golden
import test_oracle_pins as pins

PINS = [
    lambda: golden.test_oracle_tmod_update_golden("tmod_update_D1_2x2.json", oracle.update_D1),
    lambda: golden.test_oracle_tmod_update_golden("tmod_update_D1_offdiag_2x2.json", oracle.update_D1),
    lambda: golden.test_oracle_tmod_update_golden("tmod_update_D2_2x2.json", oracle.update_D2),
    lambda: golden.test_oracle_omp2d_golden("omp2d_coherent_atoms.json",
                                            golden.load("omp2d_coherent_atoms.json")["cases"][0]),
    pins.test_kronecker_identity_residual,
    lambda: pins.test_bruteforce_4x4_picks_and_coefficients(4, 4, 3),
    lambda: pins.test_bruteforce_4x4_picks_and_coefficients(6, 4, 4),
    pins.test_omp_residual_not_below_best_subset,
    pins.test_tie_rule_smallest_pair_index,
    pins.test_error_bounded_stop_and_zero_score,
    pins.test_exact_recovery_low_coherence,
    pins.test_D1_update_is_least_squares_optimum,
    pins.test_D2_update_is_least_squares_optimum,
    pins.test_closed_form_optimal_value,
    pins.test_gram_shortcut,
    pins.test_rescale_keeps_reconstruction,
    pins.test_mod_special_case,
    pins.test_iteration_monotone_updates,
    pins.test_selected_pairs_never_reselected,
]


def caught():
    """Names of the pins that fail (any exception) under the current mutant."""
    failed = []
    with np.errstate(all="ignore"):
        for fn in PINS:
            try:
                fn()
            except Exception:
                failed.append(getattr(fn, "__name__", "lambda"))
    return failed


def test_pins_pass_without_a_mutant():
    assert caught() == []


def _gram_drops_d2(D1, D2):                       # a dropped Kronecker factor
    return D1.T @ D1, np.eye(D2.shape[1])


_orig_solve = so._cholesky_solve
_orig_densify = so.densify
_orig_solve_normal = so._solve_normal
_orig_reconstruct = so.reconstruct


def _solve_perturbed(L, b):                       # an inexact least-squares re-fit
    return _orig_solve(L, b) * (1.0 + 1e-3)


def _densify_transposed(support, coef, n1, n2):  # i and j swapped (square case)
    X = _orig_densify(support, coef, n1, n2)
    return X.transpose(0, 2, 1) if n1 == n2 else X


def _solve_normal_no_normalisation(P, B, D_old):  # the atom normalisation dropped
    Dstar, D, norms, used = _orig_solve_normal(P, B, D_old)
    return Dstar, Dstar.copy(), np.ones_like(norms), used


def _reconstruct_wrong_sign(D1, D2, support, coef):  # a sign error in the model
    return -_orig_reconstruct(D1, D2, support, coef)


MUTANTS = {
    "gram_drops_d2": ("grams", _gram_drops_d2),
    "solve_perturbed": ("_cholesky_solve", _solve_perturbed),
    "densify_transposed": ("densify", _densify_transposed),
    "no_normalisation": ("_solve_normal", _solve_normal_no_normalisation),
    "reconstruct_wrong_sign": ("reconstruct", _reconstruct_wrong_sign),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_mutant_is_caught(monkeypatch, name):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(so, attr, fn)
    if hasattr(oracle, attr):
        monkeypatch.setattr(oracle, attr, fn)
    failed = caught()
    assert failed, f"no pin caught the mutant {name}"
