"""Pins of the oracle's derivative definitions (implicit function theorem on the
active set) against central finite differences of the exact LASSO solution map,
which tests/test_oracle_method.py computes by enumerating sign patterns."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_method import _brute_force_lasso, _csc_from_dense


def _problem(seed, m=14, n=7):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    lam = 0.2 * float(np.max(np.abs(A.T @ b)))
    t = rng.standard_normal(n)
    return A, b, lam, t


def _L(x, t):
    return 0.5 * float(np.sum((x - t) ** 2))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_implicit_grad_matches_finite_differences(seed):
    A, b, lam, t = _problem(seed)
    x, _ = _brute_force_lasso(A, b, lam)
    assert np.count_nonzero(x) > 0
    Ac = _csc_from_dense(A)
    db, dlam = oracle.implicit_grad(Ac, x, lam, x - t)
    rng = np.random.default_rng(100 + seed)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(A.shape[0])
        xp, _ = _brute_force_lasso(A, b + eps * d, lam)
        xm, _ = _brute_force_lasso(A, b - eps * d, lam)
        fd = (_L(xp, t) - _L(xm, t)) / (2 * eps)
        assert abs(fd - db @ d) <= 1e-6 * max(1.0, abs(fd))
    xp, _ = _brute_force_lasso(A, b, lam + eps)
    xm, _ = _brute_force_lasso(A, b, lam - eps)
    fd = (_L(xp, t) - _L(xm, t)) / (2 * eps)
    assert abs(fd - dlam) <= 1e-6 * max(1.0, abs(fd))


def test_active_set_solution_is_the_lasso_solution_on_its_support():
    A, b, lam, _ = _problem(7)
    x, _ = _brute_force_lasso(A, b, lam)
    S = np.nonzero(x)[0]
    xa = oracle.active_set_solution(_csc_from_dense(A), b, lam, S, np.sign(x[S]))
    assert np.max(np.abs(xa - x)) <= 1e-12 * max(1.0, np.max(np.abs(x)))


def test_gradient_wrt_b_lies_in_the_range_of_A_S():
    A, b, lam, t = _problem(9)
    x, _ = _brute_force_lasso(A, b, lam)
    S = np.nonzero(x)[0]
    db, _ = oracle.implicit_grad(_csc_from_dense(A), x, lam, x - t)
    # A_S^T db reproduces dL/dx on S, and db is a combination of the columns of A_S
    assert np.allclose(A[:, S].T @ db, (x - t)[S], rtol=1e-12, atol=1e-12)
    coef, res, *_ = np.linalg.lstsq(A[:, S], db, rcond=None)
    assert np.allclose(A[:, S] @ coef, db, atol=1e-12)


def test_zero_solution_has_zero_gradient():
    A, b, _, t = _problem(11)
    lam = 2.0 * float(np.max(np.abs(A.T @ b)))           # above lambda_max: x = 0
    x, _ = _brute_force_lasso(A, b, lam)
    assert np.count_nonzero(x) == 0
    db, dlam = oracle.implicit_grad(_csc_from_dense(A), x, lam, x - t)
    assert not np.any(db) and dlam == 0.0
