"""The sin^2(pi x) polynomial in objectives.cuh (Rastrigin, Ackley) against
the exact function: the constants in the kernel source, evaluated in FP32
with Horner's rule, stay within 5e-7 relative of sin^2(pi x) in FP64."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2101_06599_gb300", "csrc", "objectives.cuh")


def kernel_coefficients():
    text = open(SRC).read()
    body = text[text.index("float sin2pi(float x)"):]
    body = body[:body.index("return q * t;")]
    return [np.float32(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]


def horner32(c, x):
    x = np.asarray(x, np.float32)
    r = (x - np.rint(x)).astype(np.float32)
    t = (r * r).astype(np.float32)
    q = np.full_like(t, c[0])
    for ci in c[1:]:
        q = (q * t + ci).astype(np.float32)
    return (q * t).astype(np.float64)


def test_coefficients_match_the_fit():
    import sys
    sys.path.insert(0, os.path.dirname(SRC))
    import sin2pi_poly
    fit = np.float32(sin2pi_poly.fit())
    assert np.array_equal(np.array(kernel_coefficients(), np.float32), fit)


def test_relative_error_bound():
    c = kernel_coefficients()
    assert len(c) == 6
    x = np.concatenate([np.linspace(-30, 30, 1_000_001), np.linspace(-1e-3, 1e-3, 10001),
                        np.array([0.5, -0.5, 1.5, 29.999, 1e-30])]).astype(np.float32)
    truth = np.sin(np.pi * (x.astype(np.float64) - np.rint(x.astype(np.float64)))) ** 2
    got = horner32(c, x)
    nz = truth > 1e-30
    assert np.max(np.abs(got[nz] - truth[nz]) / truth[nz]) < 5e-7
    assert np.all(got[~nz] == 0.0)
    # integers are exact zeros, half-integers are 1 within rounding
    assert horner32(c, np.arange(-30, 31))[:].max() == 0.0
    assert np.allclose(horner32(c, np.arange(-30, 30) + 0.5), 1.0, rtol=5e-7)
