"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/pcdm_oracle.c (a dropped term,
a flipped sign, a wrong index or denominator, a sequential instead of a Jacobi
update), builds it on the CPU, points the oracle wrapper at it and runs the pin
tests of test_oracle_method.py and test_oracle_sampler.py: at least one of them
has to fail.  Nothing here touches a GPU.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as oracle_build

from . import test_oracle_glm as Glm
from . import test_oracle_method as M
from . import test_oracle_sampler as Smp
from . import test_oracle_samplings as Smv

MUTANTS = {
    "beta_denominator_n": ("double denom = (double)(n - 1 > 1 ? n - 1 : 1);",
                           "double denom = (double)(n > 1 ? n : 1);"),
    "beta_omega_not_minus_one": ("return 1.0 + (om - 1.0) * ((double)tau - 1.0) / denom;",
                                 "return 1.0 + om * ((double)tau - 1.0) / denom;"),
    "soft_threshold_sign": ("if (u < -t) return u + t;", "if (u < -t) return u - t;"),
    "gradient_sign": ("x_new = soft_threshold(x[i] - grad / bl, lambda / bl);",
                      "x_new = soft_threshold(x[i] + grad / bl, lambda / bl);"),
    "no_beta_in_threshold": ("x_new = soft_threshold(x[i] - grad / bl, lambda / bl);",
                             "x_new = soft_threshold(x[i] - grad / bl, lambda / L[i]);"),
    "L_abs_not_square": ("s += val[p] * val[p];", "s += fabs(val[p]);"),
    "omega_plus_one": ("if (count[r] > omega) omega = count[r];",
                       "if (count[r] + 1 > omega) omega = count[r] + 1;"),
    "scatter_sign": ("g[row_idx[p]] += val[p] * h;", "g[row_idx[p]] -= val[p] * h;"),
    "residual_sign_b": ("for (int64_t r = 0; r < m; ++r) g[r] = -b[r];",
                        "for (int64_t r = 0; r < m; ++r) g[r] = b[r];"),
    "gauss_seidel": ("        xbuf[t] = x_new;\n        hbuf[t] = x_new - x[i];",
                     "        xbuf[t] = x_new;\n        hbuf[t] = 0.0;\n"
                     "        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) g[row_idx[p]] += val[p] * (x_new - x[i]);\n"
                     "        x[i] = x_new;"),
    "gap_s_inverted": ("if (cinf > 0.0 && lambda / cinf < 1.0) s = lambda / cinf;",
                       "if (cinf > 0.0 && cinf / lambda < 1.0) s = cinf / lambda;"),
    "gap_drops_l1": ("terms += lambda * fabs(x[i]) + s * x[i] * c[i];", "terms += s * x[i] * c[i];"),
    "philox_multiplier": ("0xCD9E8D57u", "0xCD9E8D59u"),
    "feistel_four_rounds": ("#define ORACLE_FEISTEL_ROUNDS 12", "#define ORACLE_FEISTEL_ROUNDS 4"),
    "empty_column_keeps_x": ("            x_new = 0.0;\n        }", "            x_new = x[i];\n        }"),
    "duplicates_not_idle": ("active[j] = seen[pick] ? 0 : 1;", "active[j] = 1;"),
    "beta_du_drops_minus_one": ("(e2 / e1 - 1.0)", "(e2 / e1)"),
    "binomial_second_moment": ("*e2 = t * p_b * (1.0 + t * p_b - p_b);", "*e2 = t * p_b * (1.0 + t * p_b);"),
    "independent_pick_skewed": ("(int64_t)(((unsigned __int128)W * (unsigned __int128)(uint64_t)n) >> 64)",
                                "(int64_t)(((unsigned __int128)(W >> 1) * (unsigned __int128)(uint64_t)n) >> 64)"),
    "q_recursion_sign": ("ck -= binom * c[i];", "ck += binom * c[i];"),
}

# Mistakes planted in oracle/pcdm_oracle_glm.c (SVM dual and logistic regression).
MUTANTS_GLM = {
    "svm_L_missing_n": ("L[i] = s / (lambda * (double)n * (double)n);", "L[i] = s / (lambda * (double)n);"),
    "svm_linear_term_sign": ("return y[i] * s / (lambda * (double)n * (double)n) - 1.0 / (double)n;",
                             "return y[i] * s / (lambda * (double)n * (double)n) + 1.0 / (double)n;"),
    "svm_grad_drops_label": ("return y[i] * s / (lambda * (double)n * (double)n) - 1.0 / (double)n;",
                             "return s / (lambda * (double)n * (double)n) - 1.0 / (double)n;"),
    "svm_no_upper_clip": ("if (x_new > 1.0) x_new = 1.0;", ";"),
    "svm_empty_example_to_zero": ("                x_new = 1.0;\n            }", "                x_new = 0.0;\n            }"),
    "svm_residual_drops_label": ("const double c = problem == GLM_SVM_DUAL ? y[i] * x[i] : x[i];",
                                 "const double c = x[i];"),
    "svm_hinge_drops_label": ("const double margin = 1.0 - y[i] * wa;", "const double margin = 1.0 - wa;"),
    "svm_dual_value_sign": ("out[1] = sx / nn - uu / (2.0 * lambda * nn * nn);",
                            "out[1] = sx / nn + uu / (2.0 * lambda * nn * nn);"),
    "logistic_L_half": ("L[i] = s / 4.0;", "L[i] = s / 2.0;"),
    "logistic_grad_sign": ("s += -y[j] * val[p] / (1.0 + exp(y[j] * v[j]));",
                           "s += y[j] * val[p] / (1.0 + exp(y[j] * v[j]));"),
    "logistic_exp_sign": ("s += -y[j] * val[p] / (1.0 + exp(y[j] * v[j]));",
                          "s += -y[j] * val[p] / (1.0 + exp(-y[j] * v[j]));"),
    "logistic_regulariser_factor": ("x_new = x[i] - (grad + 2.0 * lambda * x[i]) / (beta * L[i] + 2.0 * lambda);",
                                    "x_new = x[i] - (grad + lambda * x[i]) / (beta * L[i] + lambda);"),
    "logistic_no_beta": ("x_new = x[i] - (grad + 2.0 * lambda * x[i]) / (beta * L[i] + 2.0 * lambda);",
                         "x_new = x[i] - (grad + 2.0 * lambda * x[i]) / (L[i] + 2.0 * lambda);"),
    "logistic_entropy_sign": ("ent += -alpha * softplus(t) - (1.0 - alpha) * softplus(-t);",
                              "ent += alpha * softplus(t) - (1.0 - alpha) * softplus(-t);"),
    "glm_gauss_seidel": ("        xbuf[t] = x_new;\n        hbuf[t] = x_new - x[i];",
                         "        xbuf[t] = x_new;\n        hbuf[t] = 0.0;\n"
                         "        {\n            const double c_ = problem == GLM_SVM_DUAL ? y[i] * (x_new - x[i]) : x_new - x[i];\n"
                         "            for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) v[row_idx[p]] += val[p] * c_;\n"
                         "        }\n        x[i] = x_new;"),
}

PINS_GLM = [
    Glm.test_svm_gradient_and_L_match_the_dense_dual, Glm.test_svm_gap_matches_primal_and_dual_definitions,
    Glm.test_svm_separable_full_step_is_the_exact_dual_solution,
    lambda: [Glm.test_svm_converges_to_the_brute_force_dual_solution(s) for s in (5, 6)],
    Glm.test_svm_monotone_with_conservative_beta, Glm.test_svm_empty_example_goes_to_one,
    Glm.test_svm_eso_holds_for_nice_sampling_by_enumeration,
    Glm.test_logistic_gradient_matches_finite_differences, Glm.test_logistic_L_is_the_coordinate_lipschitz_bound,
    lambda: Glm.test_logistic_converges_to_the_newton_solution(15), Glm.test_logistic_gap_is_the_scaled_gradient_norm,
    Glm.test_logistic_monotone_with_conservative_beta, Glm.test_logistic_separable_fixed_point_solves_each_coordinate,
    lambda: [Glm.test_jacobi_steps_all_start_from_the_same_point(p) for p in (oracle.SVM_DUAL, oracle.LOGISTIC)],
    lambda: [Glm.test_step_minimises_the_model_H(p, b) for p in (oracle.SVM_DUAL, oracle.LOGISTIC) for b in (1.0, 3.7)],
]

PINS = [
    M.test_beta_printed_values, M.test_L_and_omega_match_dense_definitions, M.test_dso_tightness_construction,
    M.test_eso_holds_for_nice_sampling_by_enumeration, M.test_eso_is_tight_on_the_01_matrix,
    M.test_separable_full_step_is_exact_minimiser, M.test_serial_step_minimises_along_the_coordinate,
    M.test_residual_is_maintained_exactly, M.test_monotone_with_conservative_beta,
    M.test_expected_decrease_by_enumeration, M.test_brute_force_lasso_solution, M.test_gap_record_properties,
    M.test_step_is_argmin_of_H_from_the_same_point, M.test_empty_columns_and_zero_matrix,
    M.test_objective_matches_dense,
    lambda: [Smp.test_philox_known_answers(*row) for row in Smp._kat_rows()],
    lambda: [Smp.test_every_subset_equally_likely(n, t, s) for n, t, s in [(5, 2, 2), (8, 2, 4), (10, 3, 5)]],
    Smv.test_q_values_printed_in_the_paper, Smv.test_binomial_and_nice_moments, Smv.test_independent_sampler_law,
    Smv.test_beta_du_reduces_to_nice,
    lambda: [Smv.test_independent_moments_match_the_recursion(n, t) for n, t in [(5, 3), (12, 4)]],
    lambda: [Smv.test_eso_du_holds_by_enumeration(k) for k in ("independent", "binomial")],
    Smv.test_duplicates_are_idle_in_one_iteration,
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, workdir):
    old, new = MUTANTS[name]
    src = open(oracle_build.SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    mutated = src.replace(old, new)
    c_path = os.path.join(workdir, name + ".c")
    so_path = os.path.join(workdir, name + ".so")
    with open(c_path, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", c_path,
                    oracle_build.SRC_GLM, oracle_build.SRC_THREADS, "-o", so_path, "-lm"], check=True)
    caught = []
    oracle.use_library(so_path)
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError, IndexError, KeyError, FloatingPointError):
                caught.append(getattr(pin, "__name__", "sampler pin"))
                break
    finally:
        oracle.use_library(None)
    assert caught, "no pin caught mutant " + name


@pytest.mark.parametrize("name", sorted(MUTANTS_GLM))
def test_pins_catch_glm_mutant(name, workdir):
    old, new = MUTANTS_GLM[name]
    src = open(oracle_build.SRC_GLM).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    c_path = os.path.join(workdir, "glm_" + name + ".c")
    so_path = os.path.join(workdir, "glm_" + name + ".so")
    with open(c_path, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", oracle_build.SRC,
                    c_path, oracle_build.SRC_THREADS, "-o", so_path, "-lm"], check=True)
    caught = []
    oracle.use_library(so_path)
    try:
        for pin in PINS_GLM:
            try:
                with np.errstate(all="raise"):
                    pin()
            except (AssertionError, ValueError, IndexError, KeyError, FloatingPointError, np.linalg.LinAlgError):
                caught.append(getattr(pin, "__name__", "glm pin"))
                break
    finally:
        oracle.use_library(None)
    assert caught, "no pin caught mutant " + name
