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

import pytest

import oracle
from oracle import build as oracle_build

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
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", c_path, "-o", so_path,
                    "-lm"], check=True)
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
