"""Pins of the oracle's other doubly uniform samplings (Sec. 4.1 items 4, 5)
and of beta from Theorem ESO-DU: the paper's printed law of |S|, closed forms
against the paper's recursion, sampler statistics, the ESO inequality by
exhaustive enumeration, and the idle-duplicate semantics of one iteration."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from tests.test_oracle_method import _csc_from_dense

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "q_independent_n1000_tau8.txt")


def test_q_values_printed_in_the_paper():
    q = oracle.q_independent(1000, 8)
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    for k, val in rows:
        assert round(q[int(k)], 4) == float(val)
    assert np.all(q[1:6] < 1e-5)      # "q_k ~ 0 for k = 1..5" (q_5 is about 1.04e-6)
    assert abs(q.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("n,tau", [(5, 3), (12, 4), (40, 7), (1000, 8)])
def test_independent_moments_match_the_recursion(n, tau):
    q = oracle.q_independent(n, tau)
    k = np.arange(q.size)
    e1, e2 = oracle.moments("independent", n, tau)
    assert e1 == pytest.approx(float(k @ q), rel=1e-10)
    assert e2 == pytest.approx(float((k * k) @ q), rel=1e-10)


def test_binomial_and_nice_moments():
    tau, p = 9, 0.3
    k = np.arange(tau + 1)
    q = np.array([math.comb(tau, int(j)) * p ** j * (1 - p) ** (tau - j) for j in k])
    e1, e2 = oracle.moments("binomial", 50, tau, p)
    assert e1 == pytest.approx(float(k @ q), rel=1e-12)
    assert e2 == pytest.approx(float((k * k) @ q), rel=1e-12)
    assert oracle.moments("nice", 50, tau) == (tau, tau * tau)


def test_beta_du_reduces_to_nice():
    for omega, tau, n in [(1, 5, 10), (7, 1, 30), (7, 13, 30), (100, 4096, 10**6)]:
        e1, e2 = oracle.moments("nice", n, tau)
        assert oracle.beta_du(omega, e1, e2, n) == pytest.approx(oracle.beta_nice(omega, tau, n), rel=1e-14)


def test_independent_sampler_law():
    n, tau, K = 12, 5, 20000
    q = oracle.q_independent(n, tau)
    sizes = np.zeros(tau + 1)
    incl = np.zeros(n)
    for k in range(K):
        S, act = oracle.sample_independent(7, k, n, tau)
        assert np.all((S >= 0) & (S < n))
        # the active positions are the first occurrences
        seen = set()
        for s_, a in zip(S, act):
            assert a == (s_ not in seen)
            seen.add(s_)
        sizes[act.sum()] += 1
        incl[np.unique(S)] += 1
    freq = sizes / K
    sd = np.sqrt(q * (1 - q) / K)
    assert np.all(np.abs(freq - q) <= 5 * sd + 1e-12)
    p_incl = 1 - (1 - 1 / n) ** tau
    assert np.all(np.abs(incl / K - p_incl) <= 5 * math.sqrt(p_incl * (1 - p_incl) / K))


def test_binomial_keep_frequency():
    tau, p, K = 64, 0.37, 2000
    kept = np.array([oracle.binomial_keep(3, k, tau, p).sum() for k in range(K)])
    assert kept.mean() == pytest.approx(tau * p, abs=5 * math.sqrt(tau * p * (1 - p) / K))
    assert np.all(oracle.binomial_keep(3, 0, tau, 1.0))


def _eso_sides(A, b, x, h, L, sets_with_prob, beta):
    """E f(x + h_[S]) and its ESO bound f(x) + E|S|/n (<grad f, h> + beta/2 ||h||_L^2)."""
    f = lambda v: 0.5 * float(np.sum((A @ v - b) ** 2))
    grad = A.T @ (A @ x - b)
    lhs, es = 0.0, 0.0
    for S, pr in sets_with_prob:
        hs = np.zeros_like(h)
        hs[list(S)] = h[list(S)]
        lhs += pr * f(x + hs)
        es += pr * len(S)
    n = x.size
    rhs = f(x) + es / n * (grad @ h + 0.5 * beta * float(np.sum(L * h * h)))
    return lhs, rhs


@pytest.mark.parametrize("kind", ["independent", "binomial"])
def test_eso_du_holds_by_enumeration(kind):
    rng = np.random.default_rng(5)
    m, n, tau, p = 7, 5, 3, 0.6
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6)
    A[0, :] = 1.0                                        # omega = n on row 0
    b = rng.standard_normal(m)
    L = np.maximum(np.sum(A * A, axis=0), 1e-12)
    omega = int(np.max(np.count_nonzero(A, axis=1)))
    beta = oracle.beta_sampling(omega, kind, tau, n, p)
    if kind == "independent":
        sets = [(set(t), n ** -tau) for t in itertools.product(range(n), repeat=tau)]
    else:
        sets = []
        subsets = list(itertools.combinations(range(n), tau))
        for sub in subsets:
            for keep in itertools.product((0, 1), repeat=tau):
                pr = (1 / len(subsets)) * np.prod([p if kk else 1 - p for kk in keep])
                sets.append(({s for s, kk in zip(sub, keep) if kk}, pr))
    for _ in range(20):
        x = rng.standard_normal(n)
        h = rng.standard_normal(n)
        lhs, rhs = _eso_sides(A, b, x, h, L, sets, beta)
        assert lhs <= rhs + 1e-10 * max(1.0, abs(rhs))


def test_duplicates_are_idle_in_one_iteration():
    """One tau-independent iteration equals the Jacobi step applied once to each
    distinct picked block (computed here with dense numpy)."""
    rng = np.random.default_rng(8)
    m, n = 9, 6
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    lam = 0.1
    Ac = _csc_from_dense(A)
    st = oracle.State(Ac, b, lam)
    seed, tau = 11, 5
    S, act = oracle.sample_independent(seed, 0, n, tau)
    assert (~act).any(), "choose a case with a duplicate pick"
    beta = oracle.beta_sampling(st.omega, "independent", tau, n)
    st.run_sampling("independent", tau, 1, seed, beta=beta)
    L = np.sum(A * A, axis=0)
    x = np.zeros(n)
    g = A @ x - b
    x_new = x.copy()
    for i in sorted(set(S.tolist())):
        u = x[i] - (A[:, i] @ g) / (beta * L[i])
        t = lam / (beta * L[i])
        x_new[i] = np.sign(u) * max(abs(u) - t, 0.0)
    assert np.allclose(st.x, x_new, rtol=1e-13, atol=1e-15)
    assert np.allclose(st.g, A @ x_new - b, rtol=1e-12, atol=1e-13)
