"""Pins of the oracle's tau-nice sampler against what the paper and Philox fix.

- Philox4x32-10 against the published known-answer vectors (tests/golden).
- S_k has tau distinct coordinates in [0, n) and is a pure function of (seed, k).
- A tau-nice sampling gives every tau-subset the same probability (Sec. 4.1,
  item 3): chi-square over all subsets of small ground sets.
- p_i = tau/n (eq. simple2unif), p_ij = tau(tau-1)/(n(n-1)) (eq. p_ij_equals),
  and E|J cap S|^2 (eq. 00sjs738), by frequency over many iterations.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        words = [int(w, 16) for w in lhs.split()]
        out = [int(w, 16) for w in rhs.split()]
        rows.append((words[:4], words[4:6], out))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(ctr, key, want):
    assert list(oracle.philox4x32_10(ctr, key)) == want


@pytest.mark.parametrize("n,tau", [(1, 1), (2, 1), (2, 2), (3, 2), (4, 4), (5, 3), (16, 16), (17, 9),
                                   (1000, 32), (4096, 4096), (4097, 1000), (65536, 300),
                                   (4_000_000, 2000), (500_000_000, 64), (2_147_483_647, 16)])
def test_sample_distinct_in_range(n, tau):
    for k in (0, 1, 7, 123456789):
        S = oracle.sample(0, k, n, tau)
        assert S.shape == (tau,)
        assert S.min() >= 0 and S.max() < n
        assert np.unique(S).size == tau


def test_full_sample_is_permutation():
    for n in (1, 2, 3, 10, 64, 65, 1000):
        S = oracle.sample(5, 3, n, n)
        assert sorted(S.tolist()) == list(range(n))


def test_sample_is_function_of_seed_and_k():
    a = oracle.sample(11, 5, 10_000, 200)
    assert np.array_equal(a, oracle.sample(11, 5, 10_000, 200))
    assert not np.array_equal(a, oracle.sample(11, 6, 10_000, 200))
    assert not np.array_equal(a, oracle.sample(12, 5, 10_000, 200))
    assert not np.array_equal(a, oracle.sample(11 + (1 << 32), 5, 10_000, 200))   # high key word used
    # a prefix property: tau' < tau gives the first tau' entries
    assert np.array_equal(oracle.sample(11, 5, 10_000, 50), a[:50])
    many = oracle.sample_many(11, 3, 4, 10_000, 200)
    for q in range(4):
        assert np.array_equal(many[q], oracle.sample(11, 3 + q, 10_000, 200))


def test_sample_rejects_bad_sizes():
    with pytest.raises(ValueError):
        oracle.sample(0, 0, 10, 11)
    with pytest.raises(ValueError):
        oracle.sample(0, 0, 0, 0)
    with pytest.raises(ValueError):
        oracle.sample(0, -1, 10, 1)


@pytest.mark.parametrize("n,tau,seed", [(4, 2, 1), (5, 2, 2), (6, 3, 3), (8, 2, 4), (10, 3, 5),
                                        (16, 4, 6), (17, 2, 7), (30, 2, 8)])
def test_every_subset_equally_likely(n, tau, seed):
    """Chi-square of subset frequencies against the uniform law on all C(n, tau) subsets."""
    K = 40_000
    draws = np.sort(oracle.sample_many(seed, 0, K, n, tau), axis=1)
    index = {s: q for q, s in enumerate(itertools.combinations(range(n), tau))}
    counts = np.zeros(len(index))
    for row in draws:
        counts[index[tuple(row.tolist())]] += 1
    expected = K / len(index)
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    p = stats.chi2.sf(chi2, len(index) - 1)
    assert p > 1e-5, (n, tau, chi2, p)


def test_inclusion_probability_is_tau_over_n():
    n, tau, K = 1000, 50, 8000
    draws = oracle.sample_many(21, 0, K, n, tau)
    counts = np.bincount(draws.reshape(-1), minlength=n).astype(float)
    p_i = tau / n                                     # eq. simple2unif with E|S| = tau
    expected = K * p_i
    # each count is Binomial(K, tau/n); counts are weakly dependent (sum fixed), chi-square is conservative
    chi2 = float(((counts - expected) ** 2 / (expected * (1 - p_i))).sum())
    assert stats.chi2.sf(chi2, n - 1) > 1e-5
    assert abs(counts.mean() - expected) < 1e-9


def test_pair_probability():
    n, tau, K = 40, 8, 30_000
    draws = oracle.sample_many(22, 0, K, n, tau)
    member = np.zeros((K, n), dtype=bool)
    member[np.arange(K)[:, None], draws] = True
    p_ij = tau * (tau - 1) / (n * (n - 1))            # eq. p_ij_equals for a tau-nice sampling
    worst = 0.0
    for i, j in [(0, 1), (0, 39), (5, 6), (12, 31), (38, 39), (7, 20), (2, 3), (16, 17)]:
        hits = float(np.sum(member[:, i] & member[:, j]))
        z = (hits - K * p_ij) / math.sqrt(K * p_ij * (1 - p_ij))
        worst = max(worst, abs(z))
    assert worst < 5.0


def test_intersection_second_moment_and_law():
    """|J cap S| is hypergeometric for a tau-nice S; its second moment is eq. 00sjs738."""
    n, tau, K = 60, 12, 30_000
    J = np.array([3, 10, 17, 29, 44, 58, 59])
    draws = oracle.sample_many(23, 0, K, n, tau)
    inter = np.isin(draws, J).sum(axis=1)
    sz = len(J)
    closed = sz * tau / n * (1 + (sz - 1) * (tau - 1) / max(1, n - 1))
    emp = float(np.mean(inter.astype(float) ** 2))
    se = float(np.std(inter.astype(float) ** 2)) / math.sqrt(K)
    assert abs(emp - closed) < 5 * se
    law = stats.hypergeom(n, sz, tau)
    ks = np.arange(0, sz + 1)
    counts = np.bincount(inter, minlength=sz + 1)[: sz + 1]
    probs = law.pmf(ks)
    keep = probs * K >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(probs[keep] * K, probs[~keep].sum() * K)
    if exp[-1] < 1e-9:
        obs, exp = obs[:-1], exp[:-1]
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-5


def test_large_domain_is_spread():
    """At the scale of the benchmark (n = 4e6, 2^22 Feistel domain) the sampled
    coordinates fill [0, n) evenly: chi-square over 256 equal bins, and the parity
    and residues mod 7 are balanced."""
    n, tau = 4_000_000, 65536
    S = np.concatenate([oracle.sample(99, k, n, tau) for k in range(3)])
    bins = np.bincount((S.astype(np.int64) * 256) // n, minlength=256)
    exp = S.size / 256
    assert stats.chi2.sf(float(((bins - exp) ** 2 / exp).sum()), 255) > 1e-5
    assert abs(np.mean(S % 2) - 0.5) < 5 * 0.5 / math.sqrt(S.size)
    res = np.bincount(S % 7, minlength=7)
    assert stats.chi2.sf(float(((res - S.size / 7) ** 2 / (S.size / 7)).sum()), 6) > 1e-5


def test_feistel_round_count():
    assert oracle.feistel_rounds() == 12
