"""Pins of the oracle's PCDM1 arithmetic against what the paper and the mathematics fix.

Every check computes its reference by a route independent of the oracle:
dense numpy linear algebra, exhaustive enumeration of samples or sign patterns,
or numbers printed in the paper.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import instances


# ----------------------------------------------------------------------------- helpers
def _csc_from_dense(A):
    inst = instances.from_dense(A, np.zeros(A.shape[0]), 0.0)
    return oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)


def _f(A, b, x):
    r = A @ x - b
    return 0.5 * float(r @ r)


def _F(A, b, x, lam):
    return _f(A, b, x) + lam * float(np.abs(x).sum())


def _random_sparse(rng, m, n, per_col):
    A = np.zeros((m, n))
    for i in range(n):
        rows = rng.choice(m, size=per_col, replace=False)
        A[rows, i] = rng.standard_normal(per_col)
    return A


def _tight_01(n_cols, omega):
    """0-1 matrix whose rows are all omega-subsets of the columns: every row has
    omega ones and every column the same number k of ones (Sec. 5.2, DSO tightness)."""
    rows = list(itertools.combinations(range(n_cols), omega))
    A = np.zeros((len(rows), n_cols))
    for r, cols in enumerate(rows):
        A[r, list(cols)] = 1.0
    return A


def _brute_force_lasso(A, b, lam):
    """Exact LASSO minimiser by enumerating sign patterns (n <= 8)."""
    m, n = A.shape
    best_F, best_x = math.inf, None
    for signs in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(signs, dtype=float)
        act = np.nonzero(s)[0]
        x = np.zeros(n)
        if act.size:
            As = A[:, act]
            G = As.T @ As
            if np.linalg.matrix_rank(G) < act.size:
                continue
            xa = np.linalg.solve(G, As.T @ b - lam * s[act])
            if np.any(np.sign(xa) != s[act]):
                continue
            x[act] = xa
        c = A.T @ (A @ x - b)
        off = np.setdiff1d(np.arange(n), act)
        if off.size and np.max(np.abs(c[off])) > lam * (1 + 1e-10):
            continue
        F = _F(A, b, x, lam)
        if F < best_F:
            best_F, best_x = F, x
    return best_x, best_F


# ----------------------------------------------------------------------------- beta, L, omega
def test_beta_printed_values():
    # rcv1 run (Sec. 8.3): tau = 16, omega = 291,516, n = 677,399 gives beta = 7.46 and tau/beta = 2.15
    beta = oracle.beta_nice(291_516, 16, 677_399)
    assert round(beta, 2) == 7.46
    assert round(16 / beta, 2) == 2.15
    # Table ESO: serial sampling has beta = 1, the fully parallel one beta = omega
    for om in (1, 3, 35):
        assert oracle.beta_nice(om, 1, 1000) == 1.0
        assert oracle.beta_nice(om, 1000, 1000) == pytest.approx(om, rel=0, abs=1e-12)
    # omega = 1 (separable) gives beta = 1 for every tau
    assert oracle.beta_nice(1, 500, 1000) == 1.0
    # n = 1: max(1, n-1) = 1 and tau = 1
    assert oracle.beta_nice(7, 1, 1) == 1.0
    # the billion-variable run: omega = 35, tau = 24, n = 1e9
    assert oracle.beta_nice(35, 24, 10**9) == pytest.approx(1 + 34 * 23 / (10**9 - 1), rel=1e-15)


def test_L_and_omega_match_dense_definitions():
    rng = np.random.default_rng(0)
    A = _random_sparse(rng, 30, 20, 4)
    A[:, 7] = 0.0                                   # an empty column
    Ac = _csc_from_dense(A)
    assert np.allclose(oracle.col_sqnorms(Ac), (A * A).sum(axis=0), rtol=1e-15, atol=0)
    assert oracle.omega(Ac) == int((A != 0).sum(axis=1).max())
    assert oracle.omega(_csc_from_dense(np.zeros((3, 4)))) == 0


def test_dso_tightness_construction():
    """h^T A^T A h = omega h^T D h at h = k^{-1/2} e for the 0-1 matrix of Sec. 5.2."""
    for n_cols, om in [(4, 2), (6, 3), (7, 2), (5, 5)]:
        A = _tight_01(n_cols, om)
        Ac = _csc_from_dense(A)
        L = oracle.col_sqnorms(Ac)
        k = A.sum(axis=0)[0]
        assert np.all(L == k)
        assert oracle.omega(Ac) == om
        h = np.full(n_cols, k ** -0.5)
        lhs = float(h @ A.T @ A @ h)
        rhs = oracle.omega(Ac) * float(h @ (L * h))
        assert lhs == pytest.approx(rhs, rel=1e-13)


# ----------------------------------------------------------------------------- ESO by enumeration
def _eso_sides(A, b, x, h, tau, beta, L):
    n = A.shape[1]
    grad = A.T @ (A @ x - b)
    vals = []
    for S in itertools.combinations(range(n), tau):
        hs = np.zeros(n)
        hs[list(S)] = h[list(S)]
        vals.append(_f(A, b, x + hs))
    lhs = float(np.mean(vals))
    rhs = _f(A, b, x) + tau / n * (float(grad @ h) + beta / 2 * float(np.sum(L * h * h)))
    return lhs, rhs


def test_eso_holds_for_nice_sampling_by_enumeration():
    """E f(x + h_[S]) <= f(x) + tau/n (<grad f, h> + beta/2 ||h||_L^2)  (eq. general_form_for_expectation)
    with beta from Theorem ESO-nice, exactly averaged over all tau-subsets."""
    rng = np.random.default_rng(1)
    for trial in range(6):
        m, n = 9, 7
        A = _random_sparse(rng, m, n, 1 + trial % 4)
        Ac = _csc_from_dense(A)
        L = oracle.col_sqnorms(Ac)
        om = oracle.omega(Ac)
        b = rng.standard_normal(m)
        for tau in range(1, n + 1):
            beta = oracle.beta_nice(om, tau, n)
            for _ in range(3):
                x = rng.standard_normal(n)
                h = rng.standard_normal(n)
                lhs, rhs = _eso_sides(A, b, x, h, tau, beta, L)
                assert lhs <= rhs + 1e-12 * max(1.0, abs(rhs)), (trial, tau, lhs, rhs)


def test_eso_is_tight_on_the_01_matrix():
    """On the 0-1 matrix with omega ones per row and h = e, the tau-nice ESO holds with
    equality, so any other beta (e.g. n instead of n-1 in the denominator) fails."""
    rng = np.random.default_rng(2)
    for n_cols, om in [(4, 2), (6, 3), (7, 4)]:
        A = _tight_01(n_cols, om)
        Ac = _csc_from_dense(A)
        L = oracle.col_sqnorms(Ac)
        b = rng.standard_normal(A.shape[0])
        x = rng.standard_normal(n_cols)
        h = np.ones(n_cols)
        for tau in range(1, n_cols + 1):
            beta = oracle.beta_nice(oracle.omega(Ac), tau, n_cols)
            lhs, rhs = _eso_sides(A, b, x, h, tau, beta, L)
            assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


# ----------------------------------------------------------------------------- the step
def test_separable_full_step_is_exact_minimiser():
    """omega = 1 and tau = n give beta = 1, and one step from any x solves the problem
    (Sec. 1 thought experiment; Table ESO, fully parallel row with omega = 1)."""
    rng = np.random.default_rng(3)
    m, n = 15, 5
    A = np.zeros((m, n))
    for i in range(n):
        A[3 * i:3 * i + 3, i] = rng.standard_normal(3)
    b = rng.standard_normal(m)
    Ac = _csc_from_dense(A)
    lam = 0.4 * float(np.max(np.abs(A.T @ b)))
    assert oracle.omega(Ac) == 1
    beta = oracle.beta_nice(1, n, n)
    assert beta == 1.0
    for start in (np.zeros(n), rng.standard_normal(n)):
        x = start.copy()
        g = oracle.residual(Ac, b, x)
        oracle.iteration(Ac, oracle.col_sqnorms(Ac), lam, beta, np.arange(n, dtype=np.int32), x, g)
        c = A.T @ (A @ x - b)
        on = x != 0
        assert np.all(np.abs(c[~on]) <= lam * (1 + 1e-12))
        assert np.allclose(c[on], -lam * np.sign(x[on]), rtol=0, atol=1e-12 * lam)
        assert np.any(on) and np.any(~on)


def test_serial_step_minimises_along_the_coordinate():
    """tau = 1 (serial sampling, beta = 1): the step is exact coordinate minimisation."""
    rng = np.random.default_rng(4)
    A = _random_sparse(rng, 20, 12, 5)
    b = rng.standard_normal(20)
    Ac = _csc_from_dense(A)
    L = oracle.col_sqnorms(Ac)
    lam = 0.2 * float(np.max(np.abs(A.T @ b)))
    x = rng.standard_normal(12)
    g = oracle.residual(Ac, b, x)
    for i in range(12):
        oracle.iteration(Ac, L, lam, 1.0, np.array([i], dtype=np.int32), x, g)
        c_i = float(A[:, i] @ (A @ x - b))
        if x[i] == 0:
            assert abs(c_i) <= lam * (1 + 1e-12)
        else:
            assert c_i == pytest.approx(-lam * np.sign(x[i]), abs=1e-11 * lam)


def test_residual_is_maintained_exactly():
    rng = np.random.default_rng(5)
    inst = instances.per_col_instance(80, 60, 6, nnz_star=6, seed=7)
    A = instances.dense(inst)
    st = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)
    st.run(tau=9, iters=40, seed=3)
    assert np.allclose(st.g, A @ st.x - inst.b, rtol=0, atol=1e-12 * np.abs(inst.b).max())
    assert np.any(st.x != 0)
    del rng


def test_monotone_with_conservative_beta():
    """With beta = min(omega, tau) the ESO is monotonic (Theorem proper_uniform_ESO):
    F(x_{k+1}) <= F(x_k) for every sample, not only in expectation."""
    inst = instances.per_col_instance(60, 40, 4, nnz_star=5, seed=8)
    A = instances.dense(inst)
    Ac = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    L = oracle.col_sqnorms(Ac)
    om = oracle.omega(Ac)
    for tau in (2, 8, 40):
        beta = float(min(om, tau))
        x = np.zeros(inst.n)
        g = oracle.residual(Ac, inst.b, x)
        F_prev = _F(A, inst.b, x, inst.lam)
        for k in range(150):
            oracle.iteration(Ac, L, inst.lam, beta, oracle.sample(1, k, inst.n, tau), x, g)
            F_now = _F(A, inst.b, x, inst.lam)
            assert F_now <= F_prev * (1 + 1e-13) + 1e-15, (tau, k, F_now, F_prev)
            F_prev = F_now


def test_expected_decrease_by_enumeration():
    """E F(x + h(x)_[S]) <= (1 - tau/n) F(x) + tau/n H_{beta,w}(x, h(x)) <= F(x) (eq. 1 of Sec. 5),
    averaged exactly over all tau-subsets, with beta of Theorem ESO-nice."""
    rng = np.random.default_rng(9)
    m, n = 12, 8
    A = _random_sparse(rng, m, n, 3)
    b = rng.standard_normal(m)
    Ac = _csc_from_dense(A)
    L = oracle.col_sqnorms(Ac)
    lam = 0.1 * float(np.max(np.abs(A.T @ b)))
    om = oracle.omega(Ac)
    for x0 in (np.zeros(n), rng.standard_normal(n)):
        for tau in (1, 3, 5, 8):
            beta = oracle.beta_nice(om, tau, n)
            # the full update vector h(x): the step applied to every coordinate at once
            xf, gf = x0.copy(), oracle.residual(Ac, b, x0)
            oracle.iteration(Ac, L, lam, beta, np.arange(n, dtype=np.int32), xf, gf)
            h = xf - x0
            grad = A.T @ (A @ x0 - b)
            H = _f(A, b, x0) + float(grad @ h) + beta / 2 * float(np.sum(L * h * h)) + lam * float(np.abs(x0 + h).sum())
            Fs = []
            for S in itertools.combinations(range(n), tau):
                x, g = x0.copy(), oracle.residual(Ac, b, x0)
                oracle.iteration(Ac, L, lam, beta, np.array(S, dtype=np.int32), x, g)
                Fs.append(_F(A, b, x, lam))
            EF = float(np.mean(Fs))
            F0 = _F(A, b, x0, lam)
            bound = (1 - tau / n) * F0 + tau / n * H
            assert EF <= bound + 1e-12 * abs(F0)
            assert bound <= F0 + 1e-12 * abs(F0)


def test_brute_force_lasso_solution():
    rng = np.random.default_rng(10)
    for trial in range(3):
        m, n = 10, 6
        A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.7)
        b = rng.standard_normal(m)
        lam = (0.15 + 0.1 * trial) * float(np.max(np.abs(A.T @ b)))
        x_star, F_star = _brute_force_lasso(A, b, lam)
        inst = instances.from_dense(A, b, lam)
        st = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), b, lam)
        iters, rel = st.solve(tau=3, seed=trial, rel_gap_tol=1e-13, max_iters=20000, check_every=50)
        assert rel <= 1e-13
        assert _F(A, b, st.x, lam) == pytest.approx(F_star, rel=1e-11)
        assert np.allclose(st.x, x_star, rtol=0, atol=1e-5 * np.abs(x_star).max())
        rec = oracle.gap(st.A, b, x_star, A @ x_star - b, lam)
        assert rec["gap"] <= 1e-10 * rec["primal"]


def test_gap_record_properties():
    rng = np.random.default_rng(11)
    m, n = 10, 6
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    lam = 0.3 * float(np.max(np.abs(A.T @ b)))
    _, F_star = _brute_force_lasso(A, b, lam)
    Ac = _csc_from_dense(A)
    for _ in range(20):
        x = rng.standard_normal(n) * (rng.random(n) < 0.5)
        r = A @ x - b
        rec = oracle.gap(Ac, b, x, r, lam)
        c = A.T @ r
        assert rec["primal"] == pytest.approx(_F(A, b, x, lam), rel=1e-13)
        assert rec["cinf"] == pytest.approx(np.max(np.abs(c)), rel=1e-13)
        # theta = s r is dual feasible: ||A^T theta||_inf <= lambda
        assert rec["s"] * rec["cinf"] <= lam * (1 + 1e-13)
        # weak duality around the brute-force optimum
        assert rec["dual"] <= F_star * (1 + 1e-12) + 1e-12
        assert F_star <= rec["primal"] * (1 + 1e-12)
        assert rec["gap"] >= 0
        assert rec["gap"] == pytest.approx(rec["primal"] - rec["dual"], rel=1e-9, abs=1e-12 * rec["primal"])


# ----------------------------------------------------------------------------- run bookkeeping
def test_run_is_additive_and_refresh_schedule():
    inst = instances.per_col_instance(50, 40, 5, nnz_star=4, seed=12)
    Ac = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    s1 = oracle.State(Ac, inst.b, inst.lam)
    s1.run(tau=7, iters=10, seed=4, refresh_every=3)
    s1.run(tau=7, iters=15, seed=4, refresh_every=3)
    s2 = oracle.State(Ac, inst.b, inst.lam)
    s2.run(tau=7, iters=25, seed=4, refresh_every=3)
    assert np.array_equal(s1.x, s2.x) and np.array_equal(s1.g, s2.g)
    # the same schedule by hand
    x = np.zeros(inst.n)
    g = oracle.residual(Ac, inst.b, x)
    L = oracle.col_sqnorms(Ac)
    beta = oracle.beta_nice(oracle.omega(Ac), 7, inst.n)
    for k in range(25):
        oracle.iteration(Ac, L, inst.lam, beta, oracle.sample(4, k, inst.n, 7), x, g)
        if (k + 1) % 3 == 0:
            g = oracle.residual(Ac, inst.b, x)
    assert np.array_equal(x, s2.x) and np.array_equal(g, s2.g)


def test_objective_matches_dense():
    inst = instances.per_col_instance(40, 30, 4, nnz_star=3, seed=13)
    A = instances.dense(inst)
    x = np.random.default_rng(0).standard_normal(30)
    Ac = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    assert oracle.objective(Ac, inst.b, x, inst.lam) == pytest.approx(_F(A, inst.b, x, inst.lam), rel=1e-13)


def test_empty_columns_and_zero_matrix():
    """A column with L_i = 0 takes x_i to 0 (the minimiser of lambda |x_i + t|)."""
    A = np.zeros((4, 3))
    A[1, 0] = 2.0
    b = np.array([0.0, 3.0, 0.0, 1.0])
    Ac = _csc_from_dense(A)
    L = oracle.col_sqnorms(Ac)
    x = np.array([0.0, 5.0, -2.0])
    g = oracle.residual(Ac, b, x)
    oracle.iteration(Ac, L, 0.5, 1.0, np.array([0, 1, 2], dtype=np.int32), x, g)
    assert x[1] == 0.0 and x[2] == 0.0
    assert x[0] == pytest.approx((2 * 3 - 0.5) / 4)
    assert np.allclose(g, A @ x - b)


def test_tiny_workload_converges_with_kkt():
    """The 2000 x 1000 parity workload reaches relative gap 1e-8 within 2000 iterations
    at tau = 32, and the KKT conditions of LASSO hold there."""
    inst = instances.tiny_instance()
    A = instances.dense(inst)
    st = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)
    iters, rel = st.solve(tau=32, seed=0, rel_gap_tol=1e-8, max_iters=2000, check_every=32)
    assert rel <= 1e-8, (iters, rel)
    c = A.T @ (A @ st.x - inst.b)
    on = st.x != 0
    assert np.max(np.abs(c[~on])) <= inst.lam * (1 + 1e-3)
    assert np.max(np.abs(c[on] + inst.lam * np.sign(st.x[on]))) <= 1e-3 * inst.lam


def test_step_is_argmin_of_H_from_the_same_point():
    """h(x) = argmin_h H_{beta,w}(x, h) (eq. h(x)), block by block, every block from
    the same x (Algorithm 1, step 4).  The reference minimises each one-dimensional
    H_i(t) = grad_i t + beta L_i t^2 / 2 + lambda |x_i + t| numerically."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(14)
    A = _random_sparse(rng, 25, 15, 6)
    b = rng.standard_normal(25)
    Ac = _csc_from_dense(A)
    L = oracle.col_sqnorms(Ac)
    lam = 0.15 * float(np.max(np.abs(A.T @ b)))
    beta = oracle.beta_nice(oracle.omega(Ac), 6, 15)
    for trial in range(4):
        x0 = rng.standard_normal(15) * (rng.random(15) < 0.6)
        S = rng.choice(15, size=6, replace=False).astype(np.int32)
        grad = A.T @ (A @ x0 - b)
        want = x0.copy()
        for i in S:
            Hi = lambda t, i=i: grad[i] * t + beta * L[i] * t * t / 2 + lam * abs(x0[i] + t)
            span = 10 * (abs(x0[i]) + abs(grad[i]) / (beta * L[i]) + 1)
            res = minimize_scalar(Hi, bounds=(-span, span), method="bounded",
                                  options=dict(xatol=1e-12, maxiter=2000))
            t = res.x
            if Hi(-x0[i]) <= Hi(t):                  # the kink at x_i + t = 0
                t = -x0[i]
            want[i] = x0[i] + t
        x, g = x0.copy(), oracle.residual(Ac, b, x0)
        oracle.iteration(Ac, L, lam, beta, S, x, g)
        assert np.allclose(x, want, rtol=0, atol=1e-7), (trial, np.max(np.abs(x - want)))
        assert np.allclose(g, A @ x - b, rtol=0, atol=1e-12)
