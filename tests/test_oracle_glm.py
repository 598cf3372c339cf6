"""Pins of the oracle for the SVM dual (Sec. 8.3) and L2-regularised logistic
regression (Sec. 8.4), against what the mathematics fixes: dense restatements
of the objectives, finite differences, closed-form one-step solutions,
brute-force and Newton solutions of tiny problems, strong duality and the ESO
inequality of Theorem ESO-nice by enumeration.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import instances


def _csc(inst):
    return oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)


def _rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------------------- dense restatements
def svm_dense(Ad, y, lam):
    """(f, grad f, L, P(w(x)), D(x)) of the SVM dual from the dense d x n matrix."""
    n = Ad.shape[1]
    Z = (y[:, None] * y[None, :]) * (Ad.T @ Ad)
    c = 1.0 / (lam * n * n)

    def f(x):
        return 0.5 * c * x @ Z @ x - x.sum() / n

    def grad(x):
        return c * (Z @ x) - 1.0 / n

    def primal(x):
        w = (Ad * y[None, :]) @ x / (lam * n)
        return np.maximum(0.0, 1.0 - y * (Ad.T @ w)).sum() / n + 0.5 * lam * w @ w

    return f, grad, c * np.diag(Z), primal, (lambda x: -f(x))


def logistic_dense(Ad, y, lam):
    """(F, grad f, hessian of f) of L2-regularised logistic regression."""
    def F(x):
        return np.logaddexp(0.0, -y * (Ad @ x)).sum() + lam * x @ x

    def grad(x):
        return -(Ad.T @ (y / (1.0 + np.exp(y * (Ad @ x)))))

    def hess(x):
        s = 1.0 / (1.0 + np.exp(-y * (Ad @ x)))
        return Ad.T @ ((s * (1.0 - s))[:, None] * Ad)

    return F, grad, hess


def svm_dense_instance(d, n, seed, lam=0.05, density=0.6):
    rng = _rng(seed)
    Ad = rng.standard_normal((d, n)) * (rng.random((d, n)) < density)
    for i in range(n):
        if not Ad[:, i].any():
            Ad[rng.integers(d), i] = 1.0
    y = rng.choice([-1.0, 1.0], size=n)
    return instances.labeled_from_dense(Ad, y, lam, "svm_dual"), Ad, y


def logistic_dense_instance(m, n, seed, lam=0.3, density=0.5):
    rng = _rng(seed)
    Ad = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    y = rng.choice([-1.0, 1.0], size=m)
    return instances.labeled_from_dense(Ad, y, lam, "logistic"), Ad, y


# ----------------------------------------------------------------------------- SVM dual
def test_svm_gradient_and_L_match_the_dense_dual():
    inst, Ad, y = svm_dense_instance(12, 9, seed=1)
    A = _csc(inst)
    f, grad, L, _, _ = svm_dense(Ad, y, inst.lam)
    x = _rng(2).random(inst.n)
    v = oracle.glm_residual(oracle.SVM_DUAL, A, y, x)
    np.testing.assert_allclose(oracle.glm_gradient(oracle.SVM_DUAL, A, y, v, inst.lam), grad(x), rtol=1e-12,
                               atol=1e-14)
    np.testing.assert_allclose(oracle.glm_lipschitz(oracle.SVM_DUAL, A, inst.lam), L, rtol=1e-13)
    assert oracle.glm_objective(oracle.SVM_DUAL, A, y, x, inst.lam) == pytest.approx(f(x), rel=1e-12)
    assert oracle.glm_objective(oracle.SVM_DUAL, A, y, x + 2.0, inst.lam) == np.inf   # outside the box


def test_svm_gap_matches_primal_and_dual_definitions():
    inst, Ad, y = svm_dense_instance(10, 8, seed=3)
    A = _csc(inst)
    _, _, _, primal, dual = svm_dense(Ad, y, inst.lam)
    for s in range(5):
        x = _rng(10 + s).random(inst.n)
        rec = oracle.glm_gap(oracle.SVM_DUAL, A, y, x, inst.lam)
        assert rec["primal"] == pytest.approx(primal(x), rel=1e-12)
        assert rec["dual"] == pytest.approx(dual(x), rel=1e-12, abs=1e-15)
        assert rec["gap"] >= -1e-14


def test_svm_separable_full_step_is_the_exact_dual_solution():
    # examples on disjoint features: omega = 1, tau = n gives beta = 1 and one
    # step lands on clip(lambda n / ||A_i||^2, 0, 1) for every i, the dual optimum
    d, n, lam = 12, 6, 0.02
    rng = _rng(4)
    Ad = np.zeros((d, n))
    for i in range(n):
        Ad[2 * i: 2 * i + 2, i] = rng.standard_normal(2) * (0.1 if i % 2 else 1.5)
    y = rng.choice([-1.0, 1.0], size=n)
    inst = instances.labeled_from_dense(Ad, y, lam, "svm_dual")
    st = oracle.GlmState(oracle.SVM_DUAL, _csc(inst), y, lam)
    assert st.omega == 1 and st.beta(n) == 1.0
    st.run(n, 1, seed=0)
    expect = np.clip(lam * n / (Ad * Ad).sum(axis=0), 0.0, 1.0)
    np.testing.assert_allclose(st.x, expect, rtol=1e-14)
    assert 0 < np.sum(expect == 1.0) < n          # both the clipped and the interior case occur
    assert abs(st.gap()["gap"]) <= 1e-14


def _svm_brute_force(Ad, y, lam):
    """The dual optimum of a tiny SVM by enumerating, per coordinate, the states
    {at 0, at 1, free} and keeping the state whose solution is feasible and meets
    the KKT conditions."""
    n = Ad.shape[1]
    f, grad, _, _, _ = svm_dense(Ad, y, lam)
    Z = (y[:, None] * y[None, :]) * (Ad.T @ Ad) / (lam * n * n)
    best = None
    for state in itertools.product((0, 1, 2), repeat=n):
        st = np.array(state)
        x = np.where(st == 1, 1.0, 0.0)
        F = np.nonzero(st == 2)[0]
        if F.size:
            rhs = 1.0 / n - Z[np.ix_(F, np.nonzero(st != 2)[0])] @ x[st != 2]
            x[F] = np.linalg.solve(Z[np.ix_(F, F)], rhs)
            if np.any(x[F] < -1e-12) or np.any(x[F] > 1 + 1e-12):
                continue
        g = grad(x)
        if np.any(g[st == 0] < -1e-10) or np.any(g[st == 1] > 1e-10):
            continue
        if best is None or f(x) < f(best) - 1e-15:
            best = x
    return best


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_svm_converges_to_the_brute_force_dual_solution(seed):
    inst, Ad, y = svm_dense_instance(14, 6, seed=seed, lam=0.05)
    xb = _svm_brute_force(Ad, y, inst.lam)
    assert xb is not None
    A = _csc(inst)
    assert abs(oracle.glm_gap(oracle.SVM_DUAL, A, y, xb, inst.lam)["gap"]) <= 1e-12   # strong duality
    st = oracle.GlmState(oracle.SVM_DUAL, A, y, inst.lam)
    st.run(2, 6000, seed=seed)
    np.testing.assert_allclose(st.x, xb, atol=1e-7)
    assert st.gap()["gap"] <= 1e-9


def test_svm_monotone_with_conservative_beta():
    inst = instances.svm_instance(60, 80, 6, lam=0.01, zipf=0.5, seed=8)
    A = _csc(inst)
    st = oracle.GlmState(oracle.SVM_DUAL, A, inst.y, inst.lam)
    tau = 16
    beta = float(min(st.omega, tau))
    prev = st.objective()
    for k in range(40):
        st.run(tau, 1, seed=3, beta=beta)
        cur = st.objective()
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur
    assert np.all((st.x >= 0.0) & (st.x <= 1.0))


def test_svm_empty_example_goes_to_one():
    Ad = np.array([[1.0, 0.0, 2.0], [0.5, 0.0, 0.0]])
    y = np.array([1.0, -1.0, 1.0])
    inst = instances.labeled_from_dense(Ad, y, 0.1, "svm_dual")
    st = oracle.GlmState(oracle.SVM_DUAL, _csc(inst), y, 0.1)
    assert st.L[1] == 0.0
    st.run(3, 1, seed=0)
    assert st.x[1] == 1.0


def test_svm_eso_holds_for_nice_sampling_by_enumeration():
    # Theorem ESO-nice on this f: E f(x + h_[S]) <= f(x) + (tau/n) (<grad f, h> + beta/2 ||h||_L^2)
    inst, Ad, y = svm_dense_instance(9, 7, seed=9, density=0.5)
    A = _csc(inst)
    f, grad, L, _, _ = svm_dense(Ad, y, inst.lam)
    n = inst.n
    om = oracle.omega(A)
    rng = _rng(10)
    for tau in (1, 2, 3, 5, 7):
        beta = oracle.beta_nice(om, tau, n)
        for _ in range(3):
            x, h = rng.random(n), rng.standard_normal(n)
            subsets = list(itertools.combinations(range(n), tau))
            lhs = 0.0
            for S in subsets:
                hS = np.zeros(n)
                hS[list(S)] = h[list(S)]
                lhs += f(x + hS)
            lhs /= len(subsets)
            rhs = f(x) + tau / n * (grad(x) @ h + 0.5 * beta * (L * h * h).sum())
            assert lhs <= rhs + 1e-12 * max(1.0, abs(rhs))


# ----------------------------------------------------------------------------- logistic regression
def test_logistic_gradient_matches_finite_differences():
    inst, Ad, y = logistic_dense_instance(30, 7, seed=11)
    A = _csc(inst)
    F, _, _ = logistic_dense(Ad, y, inst.lam)
    x = _rng(12).standard_normal(inst.n)
    v = oracle.glm_residual(oracle.LOGISTIC, A, y, x)
    np.testing.assert_allclose(v, Ad @ x, rtol=1e-13, atol=1e-14)
    gF = oracle.glm_gradient(oracle.LOGISTIC, A, y, v, inst.lam) + 2.0 * inst.lam * x
    eps = 1e-6
    fd = np.array([(F(x + eps * e) - F(x - eps * e)) / (2 * eps) for e in np.eye(inst.n)])
    np.testing.assert_allclose(gF, fd, rtol=1e-6, atol=1e-7)
    assert oracle.glm_objective(oracle.LOGISTIC, A, y, x, inst.lam) == pytest.approx(F(x), rel=1e-13)


def test_logistic_L_is_the_coordinate_lipschitz_bound():
    inst, Ad, y = logistic_dense_instance(40, 6, seed=13)
    A = _csc(inst)
    L = oracle.glm_lipschitz(oracle.LOGISTIC, A, inst.lam)
    np.testing.assert_allclose(L, 0.25 * (Ad * Ad).sum(axis=0), rtol=1e-13)
    F, grad, hess = logistic_dense(Ad, y, 0.0)
    rng = _rng(14)
    for _ in range(20):
        x = rng.standard_normal(inst.n) * 2
        i = int(rng.integers(inst.n))
        t = float(rng.standard_normal() * 3)
        e = np.zeros(inst.n)
        e[i] = 1.0
        assert F(x + t * e) <= F(x) + grad(x)[i] * t + 0.5 * L[i] * t * t + 1e-12
        assert hess(x)[i, i] <= L[i] * (1 + 1e-12)
    # the bound is approached where every margin is 0 (second derivative 1/4)
    np.testing.assert_allclose(np.diag(hess(np.zeros(inst.n))), L, rtol=1e-12)


def _newton(Ad, y, lam, iters=60):
    F, grad, hess = logistic_dense(Ad, y, lam)
    x = np.zeros(Ad.shape[1])
    for _ in range(iters):
        g = grad(x) + 2 * lam * x
        x = x - np.linalg.solve(hess(x) + 2 * lam * np.eye(x.size), g)
    return x


@pytest.mark.parametrize("seed", [15, 16])
def test_logistic_converges_to_the_newton_solution(seed):
    inst, Ad, y = logistic_dense_instance(50, 8, seed=seed, lam=0.2)
    xs = _newton(Ad, y, inst.lam)
    A = _csc(inst)
    assert oracle.glm_gap(oracle.LOGISTIC, A, y, xs, inst.lam)["gap"] <= 1e-12   # zero gap at the optimum
    st = oracle.GlmState(oracle.LOGISTIC, A, y, inst.lam)
    st.run(3, 4000, seed=seed)
    np.testing.assert_allclose(st.x, xs, atol=1e-8)
    assert st.gap()["gap"] <= 1e-10


def test_logistic_gap_is_the_scaled_gradient_norm():
    # at alpha_j = 1/(1 + exp(y_j z_j)) the Fenchel gap equals ||grad F||^2 / (4 lambda)
    inst, Ad, y = logistic_dense_instance(35, 9, seed=17, lam=0.7)
    A = _csc(inst)
    F, grad, _ = logistic_dense(Ad, y, inst.lam)
    for s in range(4):
        x = _rng(30 + s).standard_normal(inst.n)
        rec = oracle.glm_gap(oracle.LOGISTIC, A, y, x, inst.lam)
        gF = grad(x) + 2 * inst.lam * x
        assert rec["gap"] == pytest.approx(gF @ gF / (4 * inst.lam), rel=1e-9)
        assert rec["primal"] == pytest.approx(F(x), rel=1e-13)


def test_logistic_monotone_with_conservative_beta():
    inst = instances.logistic_instance(300, 80, 5, lam=0.5, seed=18)
    st = oracle.GlmState(oracle.LOGISTIC, _csc(inst), inst.y, inst.lam)
    tau = 20
    beta = float(min(st.omega, tau))
    prev = st.objective()
    for _ in range(30):
        st.run(tau, 1, seed=4, beta=beta)
        cur = st.objective()
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur


def test_logistic_separable_fixed_point_solves_each_coordinate():
    # omega = 1 (every example has one feature): the problem splits into n
    # one-dimensional problems; at the fixed point each coordinate's derivative vanishes
    rng = _rng(19)
    m, n, lam = 60, 6, 0.1
    Ad = np.zeros((m, n))
    Ad[np.arange(m), rng.integers(0, n, size=m)] = rng.standard_normal(m)
    y = rng.choice([-1.0, 1.0], size=m)
    inst = instances.labeled_from_dense(Ad, y, lam, "logistic")
    st = oracle.GlmState(oracle.LOGISTIC, _csc(inst), y, lam)
    assert st.omega == 1 and st.beta(n) == 1.0
    st.run(n, 200, seed=0)
    _, grad, _ = logistic_dense(Ad, y, lam)
    np.testing.assert_allclose(grad(st.x) + 2 * lam * st.x, 0.0, atol=1e-12)


@pytest.mark.parametrize("problem", [oracle.SVM_DUAL, oracle.LOGISTIC])
def test_jacobi_steps_all_start_from_the_same_point(problem):
    # Algorithm 1 computes every h_i of S_k from x_k: the joint iteration on S
    # must move each coordinate exactly as a single-coordinate iteration from x_k
    # with the same beta does, and the kept vector must then equal its definition
    if problem == oracle.SVM_DUAL:
        inst, Ad, y = svm_dense_instance(10, 8, seed=20, density=0.8)
    else:
        inst, Ad, y = logistic_dense_instance(25, 8, seed=21, density=0.8)
    A = _csc(inst)
    L = oracle.glm_lipschitz(problem, A, inst.lam)
    x0 = _rng(22).random(inst.n) * 0.5
    v0 = oracle.glm_residual(problem, A, y, x0)
    S = np.array([1, 4, 6, 2], dtype=np.int32)
    beta = 2.5
    x, v = x0.copy(), v0.copy()
    oracle.glm_iteration(problem, A, y, L, inst.lam, beta, S, x, v)
    for i in S:
        xi, vi = x0.copy(), v0.copy()
        oracle.glm_iteration(problem, A, y, L, inst.lam, beta, np.array([i], dtype=np.int32), xi, vi)
        assert x[i] == xi[i]
    assert np.array_equal(np.delete(x, S), np.delete(x0, S))
    np.testing.assert_allclose(v, oracle.glm_residual(problem, A, y, x), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("problem", [oracle.SVM_DUAL, oracle.LOGISTIC])
@pytest.mark.parametrize("beta", [1.0, 3.7])
def test_step_minimises_the_model_H(problem, beta):
    # h_i = argmin_t <grad_i f, t> + (beta L_i / 2) t^2 + Psi_i(x_i + t)  (eq. (h(x)), w = L),
    # found here by a bounded scalar minimiser on the model itself
    from scipy.optimize import minimize_scalar
    if problem == oracle.SVM_DUAL:
        inst, Ad, y = svm_dense_instance(8, 6, seed=23)
    else:
        inst, Ad, y = logistic_dense_instance(20, 6, seed=24)
    A = _csc(inst)
    L = oracle.glm_lipschitz(problem, A, inst.lam)
    rng = _rng(25)
    for i in range(inst.n):
        x0 = rng.random(inst.n) if problem == oracle.SVM_DUAL else rng.standard_normal(inst.n)
        v0 = oracle.glm_residual(problem, A, y, x0)
        gi = oracle.glm_gradient(problem, A, y, v0, inst.lam)[i]
        if problem == oracle.SVM_DUAL:
            model = lambda t: gi * t + 0.5 * beta * L[i] * t * t
            lo, hi = -x0[i], 1.0 - x0[i]
        else:
            model = lambda t: gi * t + 0.5 * beta * L[i] * t * t + inst.lam * (x0[i] + t) ** 2
            lo, hi = -50.0, 50.0
        best = minimize_scalar(model, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12}).x
        x, v = x0.copy(), v0.copy()
        oracle.glm_iteration(problem, A, y, L, inst.lam, beta, np.array([i], dtype=np.int32), x, v)
        assert x[i] - x0[i] == pytest.approx(best, abs=1e-6)   # the scalar minimiser resolves ~1e-8
