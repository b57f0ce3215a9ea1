"""Pins for the oracle's crossovers (CPU only).

- Eq. (9) as coded (smallest n with Cr^n <= U) against the literal libm
  formula min(ceil(ln U / ln Cr), D), and against exact rational Cr^n at the
  thresholds.
- The length laws of Alg. 8 (sequential exp) and NEC against the truncated
  geometric law of Eqs. (3)-(4) at D = 10 with 10^6 draws (the design of the
  paper's Fig. 2), and against each other.
- Eq. (9)'s special cases Cr = 0 and Cr = 1.
- Alg. 8's continuation test rand < Cr at the words on either side of the
  exact threshold ceil(Cr 2^32).
- The NEC segment against brute force Alg. 9 for every (D, j_rand, L), D <= 12.
- Binomial mask rate Cr + (1 - Cr) / D and the forced j_rand gene (Eq. 2).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle as O


def trunc_geom_pmf(Cr, D):
    p = np.array([Cr ** (k - 1) * (1 - Cr) for k in range(1, D)] + [Cr ** (D - 1)])
    return p


@pytest.mark.parametrize("Cr", [0.1, 0.2, 0.5, 0.9, 0.99])
def test_nec_length_matches_libm_formula(Cr):
    rng = np.random.default_rng(1)
    D = 50
    ws = rng.integers(0, 2**32, size=20000, dtype=np.uint64)
    ws[:4] = [0, 1, 2**32 - 1, 2**31]
    for w in ws:
        L = O.nec_length(int(w), Cr, D)
        U = int(w) / 2**32
        if U == 0.0:
            ref = D
        else:
            x = math.log(U) / math.log(Cr)
            if abs(x - round(x)) < 1e-9:
                continue                 # libm rounding decides; not a pin
            ref = min(math.ceil(x), D)
        assert L == ref, (w, Cr, L, ref)


@pytest.mark.parametrize("Cr", [0.1, 0.3, 0.5, 0.9])
def test_nec_length_exact_thresholds(Cr):
    """U < Cr^n  <=>  L > n, checked against exact rational powers of the FP64 Cr."""
    D = 64
    c = Fraction(Cr)
    exact_pow2 = Cr == 0.5
    for n in range(1, D):
        T = math.ceil(c ** n * 2**32)     # w < T  <=>  w / 2^32 < Cr^n
        if T < 3:
            break
        if exact_pow2:
            assert O.nec_length(T - 1, Cr, D) >= n + 1
            assert O.nec_length(T, Cr, D) <= n
        else:
            assert O.nec_length(T - 2, Cr, D) >= n + 1
            assert O.nec_length(T + 1, Cr, D) <= n


@pytest.mark.parametrize("D", [1, 2, 10, 1000])
def test_nec_length_special_cases(D):
    for w in (0, 1, 12345, 2**32 - 1):
        assert O.nec_length(w, 0.0, D) == 1
        assert O.nec_length(w, 1.0, D) == D
        assert 1 <= O.nec_length(w, 0.7, D) <= D
    assert O.nec_length(0, 0.3, D) == D          # U = 0: ln U = -inf


@pytest.mark.parametrize("Cr", [0.0, 1e-12, 0.1, 0.3, 0.5, 0.9, 0.99, 0.9999, 1.0 - 2.0**-40, 1.0])
def test_exp_continuation_at_its_threshold(Cr):
    """Alg. 8 continues iff rand < Cr: with rand = w / 2^32 that is w < T for
    T = ceil(Cr 2^32) computed exactly from the FP64 value of Cr."""
    T = math.ceil(Fraction(Cr) * 2**32)
    for w in (T - 2, T - 1, T, T + 1, 0, 1, 2**32 - 1):
        if 0 <= w < 2**32:
            assert O.exp_continues(w, Cr) == (w < T), (Cr, w, T)


@pytest.mark.parametrize("Cr", [0.1, 0.2, 0.5, 0.9])
def test_length_laws_truncated_geometric(Cr):
    D = 10
    n = 1_000_000 if Cr in (0.2, 0.9) else 200_000
    pmf = trunc_geom_pmf(Cr, D)
    # NEC: L from word 0 of stream LEN for rows i = 0 .. n-1
    nec = np.zeros(D)
    for i in range(n):
        nec[O.nec_length(O.word(7, 0, "len", 0, i, 0), Cr, D) - 1] += 1
    # sequential exp: Alg. 8 walk per row
    n_exp = n // 5
    ex = np.zeros(D)
    for i in range(n_exp):
        ex[O.exp_length(7, 0, i, Cr, D) - 1] += 1
    keep = pmf * n_exp >= 5                       # chi-square validity
    for counts, tot in ((nec, n), (ex, n_exp)):
        exp_c = pmf * tot
        k = pmf * tot >= 5
        obs = np.append(counts[k], counts[~k].sum())
        expd = np.append(exp_c[k], exp_c[~k].sum())
        if expd[-1] == 0:
            obs, expd = obs[:-1], expd[:-1]
        assert stats.chisquare(obs, expd * obs.sum() / expd.sum()).pvalue > 1e-4
    # NEC and seq-exp draw the same law (two-sample test on shared support)
    table = np.vstack([nec[keep], ex[keep]])
    assert stats.chi2_contingency(table).pvalue > 1e-4


def test_exp_length_special_cases():
    for D in (1, 5, 40):
        for i in range(20):
            assert O.exp_length(3, 0, i, 0.0, D) == 1
            assert O.exp_length(3, 0, i, 1.0, D) == D


def _alg9_segment(D, jrand, L):
    """Alg. 9 written out: copy L genes starting at j_rand, wrapping at D."""
    m = np.zeros(D, dtype=np.uint8)
    j, l = jrand, 0
    while True:
        m[j] = 1
        j = (j + 1) % D
        l += 1
        if not l < L:
            break
    return m


def test_nec_segment_is_circular_alg9():
    # brute force: every mask the oracle produced is the Alg. 9 segment, and
    # the circular test ((j - j_rand) mod D) < L reproduces all of them.
    for D in range(1, 13):
        for jrand in range(D):
            for L in range(1, D + 1):
                seg = _alg9_segment(D, jrand, L)
                circ = np.array([((j - jrand) % D) < L for j in range(D)], dtype=np.uint8)
                assert np.array_equal(seg, circ)
    for (D, Cr) in [(7, 0.8), (30, 0.9), (100, 0.5)]:
        for i in range(200):
            _, jr = O.donors(50, D, 9, 3, i)
            for xo in ("nec", "exp"):
                m, L = O.mask(D, Cr, xo, 9, 3, i, jr)
                assert np.array_equal(m, _alg9_segment(D, jr, L))


@pytest.mark.parametrize("Cr,D", [(0.1, 30), (0.5, 100), (0.9, 1000)])
def test_binomial_mask_rate(Cr, D):
    rows = 400
    tot = 0
    for i in range(rows):
        _, jr = O.donors(64, D, 5, 1, i)
        m, L = O.mask(D, Cr, "bin", 5, 1, i, jr)
        assert m[jr] == 1
        assert L == int(m.sum())
        tot += int(m.sum()) - 1                  # the non-forced genes are Bernoulli(Cr)
    n = rows * (D - 1)
    expect = Cr * n
    sd = math.sqrt(n * Cr * (1 - Cr))
    assert abs(tot - expect) < 5 * sd
    rate = (tot + rows) / (rows * D)
    assert abs(rate - (Cr + (1 - Cr) / D)) < 5 * sd / (rows * D)


def test_binomial_special_cases():
    D = 33
    for i in range(30):
        _, jr = O.donors(64, D, 5, 1, i)
        m0, _ = O.mask(D, 0.0, "bin", 5, 1, i, jr)
        assert m0.sum() == 1 and m0[jr] == 1
        m1, _ = O.mask(D, 1.0, "bin", 5, 1, i, jr)
        assert m1.sum() == D
