"""Pins of the oracle's base index rules (Alg. 3-6 and DE/best/1) against
what their definitions fix: the support and uniformity of each index, the
per-generation offset shared by every row, the bijection of the permutation
rule, the exclusions of the best rule."""
import numpy as np
import pytest
from scipy import stats

import oracle as O


def chi2_uniform(counts):
    counts = np.asarray(counts, dtype=np.float64)
    exp = np.full_like(counts, counts.sum() / counts.size)
    return stats.chisquare(counts, exp).pvalue


def test_random_base_is_uniform_over_all_rows():
    """Alg. 3 (read as r0 = floor(N rand)): every row, the row itself
    included, equally likely; Alg. 6: r1 != r0 and r2 != r1, each offset
    uniform in [1, N - 1]."""
    N, D, seed = 7, 5, 3
    c0 = np.zeros(N)
    c1 = np.zeros(N - 1)
    c2 = np.zeros(N - 1)
    for g in range(2000):
        for i in range(N):
            (r0, r1, r2), j = O.donors_base(N, D, seed, g, i, "random")
            assert 0 <= r0 < N and r1 != r0 and r2 != r1 and 0 <= j < D
            c0[r0] += 1
            c1[(r1 - r0) % N - 1] += 1
            c2[(r2 - r1) % N - 1] += 1
    assert chi2_uniform(c0) > 1e-4
    assert chi2_uniform(c1) > 1e-4 and chi2_uniform(c2) > 1e-4


def test_offset_base_is_one_offset_per_generation():
    """Alg. 4: r0 = (i + r_g) mod N with the same r_g in [1, N - 1] for every
    row of a generation; over generations r_g is uniform."""
    N, seed = 9, 11
    counts = np.zeros(N - 1)
    for g in range(4000):
        offs = {(O.donors_base(N, 4, seed, g, i, "offset")[0][0] - i) % N for i in range(N)}
        assert len(offs) == 1
        off = offs.pop()
        assert 1 <= off <= N - 1 and off == O.base_offset(N, seed, g)
        counts[off - 1] += 1
    assert chi2_uniform(counts) > 1e-4


@pytest.mark.parametrize("N", [4, 5, 7, 16, 17, 100, 255, 256, 257, 1000, 4097])
def test_permutation_base_is_a_bijection(N):
    """Alg. 5: the base rows of one generation are a permutation of the rows."""
    for g in (0, 1, 77):
        perm = [O.base_perm(N, 5, g, i) for i in range(N)]
        assert sorted(perm) == list(range(N))


def test_permutation_base_changes_and_is_uniform_over_generations():
    N, seed = 8, 2
    seen = set()
    counts = np.zeros((N, N))
    for g in range(4000):
        perm = tuple(O.base_perm(N, seed, g, i) for i in range(N))
        seen.add(perm)
        for i, r in enumerate(perm):
            counts[i, r] += 1
    assert len(seen) > 3000                      # distinct permutations across generations
    for i in range(N):                           # each row's base row uniform over the rows
        assert chi2_uniform(counts[i]) > 1e-4


def test_best_base_excludes_row_and_best():
    """DE/best/1: r0 is the given best row; r1, r2 distinct, neither the row
    nor the best row, and uniform over what is left."""
    N, D, seed, best = 6, 3, 8, 2
    counts = {i: np.zeros(N) for i in range(N)}
    for g in range(3000):
        for i in range(N):
            (r0, r1, r2), _ = O.donors_base(N, D, seed, g, i, "best", best=best)
            assert r0 == best
            assert len({i, best, r1, r2}) == (4 if i != best else 3)
            counts[i][r1] += 1
    for i in range(N):
        allowed = [k for k in range(N) if k != i and k != best]
        assert chi2_uniform(counts[i][allowed]) > 1e-4
        assert counts[i][i] == 0 and counts[i][best] == 0


def test_distinct_rule_unchanged_and_jrand_shared():
    """The default rule is the distinct-donor rule; every rule draws j_rand
    from the same word, so the crossover masks do not depend on the rule."""
    for g in range(50):
        for i in range(10):
            d, j = O.donors(10, 13, 4, g, i)
            assert O.donors_base(10, 13, 4, g, i, "distinct") == (d, j)
            for base in ("random", "offset", "permutation", "best"):
                assert O.donors_base(10, 13, 4, g, i, base, best=3)[1] == j


def test_best_rule_step_uses_the_argmin_row():
    """One oracle step with the best rule: every trial's unmasked genes are
    its parent's, and with Cr = 1 and F = 0 every trial is the best row."""
    N, D = 12, 6
    pop = O.init(N, D, -5.0, 5.0, 9)
    fit = O.evaluate("sphere", pop)
    b = O.argmin(fit)
    s = O.step(pop, fit, 0.0, 1.0, "nec", "sphere", -5.0, 5.0, 9, 0, base="best")
    assert np.all(s.draws[:, 0] == b)
    assert np.array_equal(s.trial, np.repeat(pop[b][None, :], N, axis=0))
