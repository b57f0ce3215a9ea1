"""Pins for the oracle's random draws (CPU only).

- Philox4x32-10 against the generator authors' known-answer vectors.
- Donor indices: distinct, != i, uniform over ordered triples (exhaustive
  chi-square at tiny N).
- j_rand uniform over [0, D).
- Initial population: inside the box, on the 2^-24 grid, uniform.
"""
import os
from itertools import permutations

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLD) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key) == out


def test_philox_word_layout():
    # word idx of a stream is word idx&3 of the block at counter (idx>>2, i, g, stream<<24|inst)
    seed = 0x0123456789ABCDEF
    for (stream, g, i, idx, inst) in [(1, 0, 0, 0, 0), (3, 7, 5, 13, 2), (4, 2**31 + 5, 99, 6, 0xABCDEF)]:
        blk = O.philox([idx >> 2, i, g & 0xFFFFFFFF, (stream << 24) | inst],
                       [seed & 0xFFFFFFFF, seed >> 32])
        assert O.word(seed, inst, stream, g, i, idx) == blk[idx & 3]


@pytest.mark.parametrize("N", [4, 5, 8])
def test_donors_uniform_over_ordered_triples(N):
    D = 7
    i = N // 2
    triples = [t for t in permutations([k for k in range(N) if k != i], 3)]
    index = {t: n for n, t in enumerate(triples)}
    counts = np.zeros(len(triples))
    jr = np.zeros(D)
    draws = 200 * len(triples)
    for g in range(draws):
        r, j = O.donors(N, D, seed=11, g=g, i=i)
        assert len(set(r)) == 3 and i not in r
        assert all(0 <= v < N for v in r)
        counts[index[r]] += 1
        jr[j] += 1
    assert stats.chisquare(counts).pvalue > 1e-4
    assert stats.chisquare(jr).pvalue > 1e-4


def test_donors_distinct_many_rows():
    for N in (4, 6, 100, 1024):
        for i in range(0, N, max(1, N // 37)):
            for g in range(5):
                r, j = O.donors(N, 13, seed=3, g=g, i=i)
                assert len({i, *r}) == 4
                assert 0 <= j < 13


def test_init_box_grid_and_uniformity():
    N, D = 64, 50
    pop = O.init(N, D, 0.0, 1.0, seed=5)
    assert pop.min() >= 0.0 and pop.max() <= 1.0
    scaled = pop.astype(np.float64) * 2**24
    assert np.all(scaled == np.floor(scaled))          # (w >> 8) * 2^-24 exactly
    assert stats.kstest(pop.ravel(), "uniform").pvalue > 1e-4
    pop2 = O.init(N, D, -5.12, 5.12, seed=5)
    assert pop2.min() >= np.float32(-5.12) and pop2.max() <= np.float32(5.12)
    # mean of U[-a, a] is 0 and its std a / sqrt(3); 5-sigma bounds for n samples
    n = pop2.size
    sd = 5.12 / np.sqrt(3)
    assert abs(pop2.mean()) < 5 * sd / np.sqrt(n)
    assert abs(pop2.std() - sd) < 5 * sd / np.sqrt(n)


def test_init_depends_on_seed_and_instance():
    a = O.init(8, 8, -1, 1, seed=1)
    b = O.init(8, 8, -1, 1, seed=2)
    c = O.init(8, 8, -1, 1, seed=1, inst=1)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(a, O.init(8, 8, -1, 1, seed=1))
