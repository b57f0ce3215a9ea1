"""Pins for the oracle's best-row rule (CPU only).

The paper reports the best value and the generation it was reached (Tables
III-V) but says nothing about ties or non-finite values. The readings used
on both sides: the best row is the one of least fitness, the lowest index
among equal values (a later row must be strictly better to take over, as in
the strict '<' selection of Alg. 1), and a NaN fitness counts as +inf, so it
is never preferred to a finite value, and an all-NaN population names row 0.

Every expectation below is written out by hand; none is computed by another
argmin (numpy's argmin, for one, prefers NaN to any number).
"""
import math

import numpy as np
import pytest

import oracle as O

NAN = float("nan")
INF = float("inf")

CASES = [
    # (fitness values, expected row)
    ([3.0], 0),
    ([5.0, 4.0, 3.0, 2.0, 1.0], 4),
    ([1.0, 2.0, 3.0], 0),
    ([2.0, 1.0, 1.0, 1.0], 1),                 # ties: the lowest index
    ([0.0, -0.0, 0.0], 0),                      # +0 and -0 compare equal
    ([-0.0, 0.0], 0),
    ([7.0, 7.0, 7.0, 7.0], 0),
    ([NAN, 5.0, 2.0], 2),                       # NaN never wins against a number
    ([NAN, INF, 1e300], 2),
    ([2.0, NAN, 2.0, NAN], 0),
    ([NAN, NAN, NAN], 0),                       # all NaN: row 0
    ([NAN, INF], 0),                            # NaN and +inf are equal: the first
    ([INF, NAN], 0),
    ([INF, INF, 3.0], 2),
    ([-INF, -1e308, -INF], 0),
    ([1.0, 1.0 - 2.0 ** -52, 1.0], 1),          # one ulp below 1 is strictly better
    ([1.0, 1.0 + 2.0 ** -52, 1.0], 0),
    ([1e-320, 5e-324, 0.0], 2),                 # subnormals order like any number
]


@pytest.mark.parametrize("fit,want", CASES)
def test_argmin_hand_cases(fit, want):
    assert O.argmin(np.array(fit, dtype=np.float64)) == want


def test_argmin_lowest_index_over_every_tie_pattern():
    """All 3^5 arrays over {1, 2, NaN}: the answer is the first position of
    the least non-NaN value, else 0, read off position by position."""
    vals = [1.0, 2.0, NAN]
    for code in range(3 ** 5):
        a, c = [], code
        for _ in range(5):
            a.append(vals[c % 3])
            c //= 3
        if 1.0 in a:
            want = a.index(1.0)
        elif 2.0 in a:
            want = a.index(2.0)
        else:
            want = 0
        assert O.argmin(np.array(a)) == want, a


def test_argmin_is_not_numpys_nan_rule():
    a = np.array([NAN, 1.0])
    assert int(np.argmin(a)) == 0          # numpy picks the NaN
    assert O.argmin(a) == 1
    assert math.isnan(a[0])
