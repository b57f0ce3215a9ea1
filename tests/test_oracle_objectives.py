"""Pins for the oracle's FP64 objectives (CPU only): closed-form optima from
Section 4 (Ackley f(0) = 0, Griewank f(0) = 0, Rosenbrock f(1) = 0), values
at integer points and on coordinate axes, the shifted-rotated forms at the
shift and along rotated axes, and the orthogonality of the seeded rotation."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import workloads as W

DS = [1, 2, 7, 30, 1000]


@pytest.mark.parametrize("D", DS)
def test_optima_are_zero(D):
    z = np.zeros(D, np.float32)
    for obj in ("sphere", "rastrigin", "ackley", "griewank", "elliptic"):
        assert abs(O.evaluate(obj, z)) < 1e-12, obj
    assert O.evaluate("rosenbrock", np.ones(D, np.float32)) == 0.0


@pytest.mark.parametrize("D", DS)
def test_integer_points(D):
    rng = np.random.default_rng(D)
    k = rng.integers(-5, 6, size=D).astype(np.float32)
    # cos(2 pi k) = 1 at integers: Rastrigin reduces to the sphere
    assert O.evaluate("rastrigin", k) == pytest.approx(float((k.astype(np.float64) ** 2).sum()), abs=1e-9)
    assert O.evaluate("sphere", k) == float((k.astype(np.float64) ** 2).sum())
    # Rosenbrock: f(0) = D - 1 and f(2,...,2) = 401 (D - 1)
    assert O.evaluate("rosenbrock", np.zeros(D, np.float32)) == D - 1
    assert O.evaluate("rosenbrock", np.full(D, 2, np.float32)) == 401 * (D - 1)


@pytest.mark.parametrize("b", [0.2, 0.02])
@pytest.mark.parametrize("D", [1, 5, 100])
def test_ackley_on_integer_diagonal(b, D):
    # x = (k, ..., k): mean x^2 = k^2 and cos(2 pi k) = 1, so f = 20 (1 - exp(-b |k|))
    for k in (1, 2, -3):
        x = np.full(D, k, np.float32)
        assert O.evaluate("ackley", x, ackley_b=b) == pytest.approx(20 * (1 - math.exp(-b * abs(k))), rel=1e-12)


def test_griewank_single_axis():
    D = 9
    for j in range(D):
        for a in (1.5, -37.25, 300.0):
            x = np.zeros(D, np.float32)
            x[j] = a
            ref = a * a / 4000 - math.cos(a / math.sqrt(j + 1)) + 1     # other factors are cos 0 = 1
            assert O.evaluate("griewank", x) == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_elliptic_axes():
    D = 11
    for j in range(D):
        x = np.zeros(D, np.float32)
        x[j] = 1.0
        assert O.evaluate("elliptic", x) == pytest.approx(10 ** (6 * j / (D - 1)), rel=1e-12)
    assert O.evaluate("elliptic", np.array([3.0], np.float32)) == 9.0


def test_rotation_is_orthogonal():
    for D in (2, 16, 128):
        q = W.rotation(D, seed=3, dtype=np.float64)
        assert np.abs(q.T @ q - np.eye(D)).max() < 1e-12
        q2 = W.rotation(D, seed=3, dtype=np.float64)
        assert np.array_equal(q, q2)


def test_shifted_rotated_at_shift_and_axes():
    D = 16
    o = W.shift_vector(D, seed=2)
    R = W.rotation(D, seed=3)
    for obj in ("sr_rastrigin", "sr_elliptic"):
        assert abs(O.evaluate(obj, o, shift=o, rot=R)) < 1e-9
    # identity rotation: plain objective of x - o
    I = np.eye(D, dtype=np.float32)
    x = W.population(3, D, -100, 100, seed=1)
    zero = np.zeros(D, np.float32)
    for row in x:
        d = (row.astype(np.float64) - o.astype(np.float64)).astype(np.float32)
        assert O.evaluate("sr_rastrigin", row, shift=o, rot=I) == pytest.approx(O.evaluate("rastrigin", d), rel=1e-6)
    # along the k-th rotated axis (x = t R[k, :], o = 0): z = t e_k
    for k in (0, 5, D - 1):
        t = 3.0
        x = (t * R[k, :].astype(np.float64)).astype(np.float32)
        ref = 10 ** (6 * k / (D - 1)) * t * t
        assert O.evaluate("sr_elliptic", x, shift=zero, rot=R) == pytest.approx(ref, rel=1e-5)


def test_shifted_rotated_at_rotated_integer_points():
    """x = o + R^T n with n an integer vector gives z = n, so the rotated
    Rastrigin is sum n_k^2 (every cosine is 1) and the rotated elliptic is
    sum 10^(6k/(D-1)) n_k^2: pins the direction of the rotation, the sign of
    the shift and the index of each weight."""
    D = 12
    o = W.shift_vector(D, seed=2).astype(np.float64)
    R = W.rotation(D, seed=3, dtype=np.float64)
    rng = np.random.default_rng(5)
    for _ in range(4):
        n = rng.integers(-5, 6, size=D).astype(np.float64)
        x = o + R.T @ n
        w = 10.0 ** (6.0 * np.arange(D) / (D - 1))
        x32 = x.astype(np.float32)                 # the oracle takes FP32 inputs: z = n + O(1e-5)
        f_r = O.evaluate("sr_rastrigin", x32, shift=o.astype(np.float32), rot=R.astype(np.float32))
        f_e = O.evaluate("sr_elliptic", x32, shift=o.astype(np.float32), rot=R.astype(np.float32))
        assert f_r == pytest.approx((n * n).sum(), rel=1e-3, abs=1e-2)
        assert f_e == pytest.approx((w * n * n).sum(), rel=1e-4, abs=1e-2)


def test_shifted_rotated_with_a_permutation():
    """R a permutation matrix: z_k = x_pi(k) - o_pi(k), so the elliptic weight
    of row k applies to gene pi(k)."""
    D = 9
    pi = np.array([3, 0, 8, 1, 5, 2, 7, 4, 6])
    P = np.zeros((D, D), np.float32)
    P[np.arange(D), pi] = 1.0
    o = W.shift_vector(D, seed=2)
    x = W.population(2, D, -100, 100, seed=4)
    w = 10.0 ** (6.0 * np.arange(D) / (D - 1))
    for row in x:
        a = row.astype(np.float64) - o.astype(np.float64)
        ref = (w * a[pi] ** 2).sum()
        assert O.evaluate("sr_elliptic", row, shift=o, rot=P) == pytest.approx(ref, rel=1e-12)


def test_rosenbrock_pair_order():
    # f(x0, x1) = 100 (x0^2 - x1)^2 + (1 - x0)^2: (2, 0) -> 1601, (0, 2) -> 401
    assert O.evaluate("rosenbrock", np.array([2.0, 0.0], np.float32)) == 1601.0
    assert O.evaluate("rosenbrock", np.array([0.0, 2.0], np.float32)) == 401.0
    # D = 3 chains the pairs (0,1) and (1,2): (1, 1, 3) -> 0 + 100 * 4 = 400
    assert O.evaluate("rosenbrock", np.array([1.0, 1.0, 3.0], np.float32)) == 400.0
