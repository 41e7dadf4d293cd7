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


# ------------------------------------------------- the extensions' oracles
import test_oracle_denoise as pins_dn  # noqa: E402
import test_oracle_mlp as pins_mlp  # noqa: E402
import test_oracle_ortho as pins_or  # noqa: E402
import test_oracle_tmod3 as pins_t3  # noqa: E402
from oracle import denoise as o_dn  # noqa: E402
from oracle import mlp as o_mlp  # noqa: E402
from oracle import ortho as o_or  # noqa: E402
from oracle import tmod3 as o_t3  # noqa: E402

_orig_polar = o_or._polar
_orig_unfold = o_t3.unfold
_orig_gelu_grad = o_mlp.gelu_grad


def _polar_without_vt(B):                         # U alone instead of U V^T
    U, S, Vt = np.linalg.svd(B)
    return U, S


def _unfold_row_major(T, k):                      # the other column order
    return np.moveaxis(T, k, 0).reshape(T.shape[k], -1, order="C")


def _gelu_grad_no_density_term(u):               # Phi(u) only, the u phi(u) term dropped
    import math
    from scipy.special import erf
    return 0.5 * (1.0 + erf(u / math.sqrt(2.0)))


def _average_without_counts(patches, H, W):      # sums instead of averages
    N, p, _ = patches.shape
    acc = np.zeros((H, W))
    k = 0
    for r in range(H - p + 1):
        for c in range(W - p + 1):
            acc[r:r + p, c:c + p] += patches[k]
            k += 1
    return acc


EXT_MUTANTS = {
    "procrustes_without_vt": (o_or, "_polar", _polar_without_vt, [
        lambda: pins_or.test_procrustes_beats_every_other_orthonormal_dictionary(1),
        lambda: pins_or.test_procrustes_beats_every_other_orthonormal_dictionary(2),
        lambda: pins_or.test_procrustes_recovers_a_planted_dictionary(1),
        pins_or.test_ortho_iteration_is_monotone_and_orthonormal,
        golden.test_oracle_threshold_and_procrustes_golden]),
    "unfolding_row_major": (o_t3, "unfold", _unfold_row_major, [
        pins_t3.test_unfolding_identity,
        lambda: pins_t3.test_mode_update_is_least_squares_optimum(0),
        lambda: pins_t3.test_mode_update_is_least_squares_optimum(2),
        golden.test_oracle_tmod3_update_golden]),
    "gelu_grad_without_density": (o_mlp, "gelu_grad", _gelu_grad_no_density_term, [
        lambda: pins_mlp.test_gradients_match_central_differences("W1"),
        pins_mlp.test_gelu_definition_and_derivative,
        golden.test_oracle_mlp_golden]),
    "average_without_counts": (o_dn, "patch_average", _average_without_counts, [
        pins_dn.test_average_of_exact_patches_is_the_image,
        pins_dn.test_average_weights_by_brute_force,
        golden.test_oracle_denoise_golden]),
}


@pytest.mark.parametrize("name", sorted(EXT_MUTANTS))
def test_every_extension_mutant_is_caught(monkeypatch, name):
    mod, attr, fn, pin_list = EXT_MUTANTS[name]
    with np.errstate(all="ignore"):
        for p in pin_list:                         # every pin passes on the real oracle
            p()
    monkeypatch.setattr(mod, attr, fn)
    failed = 0
    with np.errstate(all="ignore"):
        for p in pin_list:
            try:
                p()
            except Exception:
                failed += 1
    assert failed, f"no pin caught the mutant {name}"
