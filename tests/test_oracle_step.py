"""Pins for the oracle's generation step (CPU only).

- Alg. 1 (the oracle: mutate, recombine, evaluate, select row by row) and
  Alg. 2 (crossover mask first, mutation only on masked genes, one where())
  give the same population: the paper states the two are equivalent. Alg. 2
  is written here with numpy from the oracle's draws.
- Exact mutation on a population of small integers (Eq. 1 with r1 the base
  and r2 - r3 the difference).
- Cr = 1 makes bin, exp and NEC identical; Cr = 0 makes exp and NEC
  identical and changes only gene j_rand; F = 0 copies the base donor.
- Invariants over a run: per-row fitness never increases, the population
  stays in the box, unmasked genes are the parent's, ties keep the parent.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import workloads as W


def _setup(N, D, obj, seed=1):
    lo, hi = W.BOXES[obj]
    pop = W.population(N, D, lo, hi, seed)
    fit = O.evaluate(obj, pop)
    return pop, fit, lo, hi


def _alg2(pop, fit, s, F, Cr, xo, obj, lo, hi, seed, g):
    """Alg. 2 with numpy: mask first, u = x copied, masked genes mutated."""
    N, D = pop.shape
    r = s.r
    jr = s.jrand
    if xo == "bin":
        mask = np.zeros((N, D), bool)
        for i in range(N):
            for j in range(D):
                w = O.word(seed, 0, "bin", g, i, j)
                mask[i, j] = (w / 2**32 < Cr) or j == jr[i]
    else:
        j = np.arange(D)[None, :]
        mask = ((j - jr[:, None]) % D) < s.L[:, None]
    u = pop.copy()
    x1, x2, x3 = pop[r[:, 0]], pop[r[:, 1]], pop[r[:, 2]]
    v = x1 + np.float32(F) * (x2 - x3)                 # float32 numpy ops, one rounding each
    v = np.clip(v, np.float32(lo), np.float32(hi))
    u[mask] = v[mask]
    fu = O.evaluate(obj, u)
    idx = np.where(fu < fit)[0]
    new = pop.copy()
    new[idx] = u[idx]
    newfit = fit.copy()
    newfit[idx] = fu[idx]
    return u, mask, new, newfit


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("obj,N,D,Cr", [("sphere", 20, 30, 0.9), ("rastrigin", 17, 33, 0.3),
                                        ("rosenbrock", 12, 9, 0.5), ("ackley", 9, 50, 0.95)])
def test_alg1_equals_alg2(xo, obj, N, D, Cr):
    pop, fit, lo, hi = _setup(N, D, obj)
    F, seed, g = 0.5, 77, 3
    s = O.step(pop, fit, F, Cr, xo, obj, lo, hi, seed, g, want_mask=True)
    u, mask, new, newfit = _alg2(pop, fit, s, F, Cr, xo, obj, lo, hi, seed, g)
    assert np.array_equal(mask, s.mask.astype(bool))
    assert np.array_equal(u.view(np.uint32), s.trial.view(np.uint32))
    assert np.array_equal(new.view(np.uint32), s.pop.view(np.uint32))
    assert np.array_equal(newfit, s.fit)


def test_mutation_exact_on_integer_population():
    N, D = 10, 12
    pop = np.repeat(np.arange(N, dtype=np.float32)[:, None], D, axis=1)   # row k is all k
    fit = np.full(N, np.inf)
    s = O.step(pop, fit, 0.5, 1.0, "bin", "sphere", -100, 100, seed=4, g=0)
    for i in range(N):
        r1, r2, r3 = s.r[i]
        expect = r1 + 0.5 * (r2 - r3)                  # exact in binary32
        assert np.all(s.trial[i] == np.float32(expect))


def test_mutation_clips_to_box():
    N, D = 10, 12
    pop = np.repeat(np.arange(N, dtype=np.float32)[:, None], D, axis=1)
    fit = np.full(N, np.inf)
    s = O.step(pop, fit, 3.0, 1.0, "nec", "sphere", 0.0, 9.0, seed=4, g=0)
    for i in range(N):
        r1, r2, r3 = s.r[i]
        expect = min(max(r1 + 3.0 * (r2 - r3), 0.0), 9.0)
        assert np.all(s.trial[i] == np.float32(expect))


@pytest.mark.parametrize("xo", ["bin", "nec"])
def test_midpoint_repair_on_integer_population(xo):
    """Midpoint repair: a mutant gene below lo becomes the point halfway
    between lo and the target gene (equal distances, exact on this integer
    population), above hi halfway between hi and the target; genes whose
    mutant is inside the box are the mutant, genes outside the mask are the
    parent, and the only differences from clipping are at the repaired
    genes."""
    N, D, lo, hi, F = 10, 12, 0.0, 9.0, 3.0
    pop = np.repeat(np.arange(N, dtype=np.float32)[:, None], D, axis=1)   # row k is all k
    pop[:, ::3] = (9 - np.arange(N, dtype=np.float32))[:, None]           # a second column pattern
    fit = np.full(N, np.inf)
    s = O.step(pop, fit, F, 0.7, xo, "sphere", lo, hi, seed=4, g=0, want_mask=True, repair="midpoint")
    c = O.step(pop, fit, F, 0.7, xo, "sphere", lo, hi, seed=4, g=0, want_mask=True, repair="clip")
    assert np.array_equal(s.mask, c.mask) and np.array_equal(s.draws, c.draws)
    below = above = 0
    for i in range(N):
        r1, r2, r3 = s.r[i]
        for j in range(D):
            u, x = float(s.trial[i, j]), float(pop[i, j])
            if not s.mask[i, j]:
                assert u == x
                continue
            v = float(pop[r1, j]) + F * (float(pop[r2, j]) - float(pop[r3, j]))   # Eq. 1, exact here
            if v < lo:
                below += 1
                assert u - lo == x - u and lo <= u <= x
                assert float(c.trial[i, j]) == lo
            elif v > hi:
                above += 1
                assert hi - u == u - x and x <= u <= hi
                assert float(c.trial[i, j]) == hi
            else:
                assert u == v == float(c.trial[i, j])
    assert below > 0 and above > 0


def test_cr_one_and_zero_identities():
    N, D, obj = 16, 25, "rastrigin"
    pop, fit, lo, hi = _setup(N, D, obj)
    t = {xo: O.step(pop, fit, 0.7, 1.0, xo, obj, lo, hi, 5, 2) for xo in ("bin", "exp", "nec")}
    assert np.array_equal(t["bin"].trial, t["exp"].trial)
    assert np.array_equal(t["bin"].trial, t["nec"].trial)
    assert np.all(t["nec"].L == D) and np.all(t["exp"].L == D)
    z = {xo: O.step(pop, fit, 0.7, 0.0, xo, obj, lo, hi, 5, 2, want_mask=True) for xo in ("bin", "exp", "nec")}
    assert np.array_equal(z["exp"].trial, z["nec"].trial)
    for xo in ("bin", "exp", "nec"):
        m = z[xo].mask.astype(bool)
        assert np.all(m.sum(1) == 1)
        assert np.all(m[np.arange(N), z[xo].jrand])
        assert np.array_equal(z[xo].trial[~m], pop[~m])


def test_f_zero_copies_base_donor():
    N, D, obj = 16, 25, "sphere"
    pop, fit, lo, hi = _setup(N, D, obj)
    s = O.step(pop, fit, 0.0, 0.6, "bin", obj, lo, hi, 5, 2, want_mask=True)
    m = s.mask.astype(bool)
    for i in range(N):
        assert np.array_equal(s.trial[i][m[i]], pop[s.r[i, 0]][m[i]])


def test_ties_keep_parent():
    N, D = 8, 10
    pop = np.tile(W.population(1, D, -5, 5, 3), (N, 1))     # identical rows: every trial equals its parent
    fit = O.evaluate("rastrigin", pop)
    s = O.step(pop, fit, 0.5, 0.9, "nec", "rastrigin", -5.12, 5.12, 1, 0)
    assert np.array_equal(s.trial, pop)
    assert not s.accept.any()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_run_invariants_and_progress(xo):
    N, D, obj = 30, 10, "sphere"
    lo, hi = W.BOXES[obj]
    pop = O.init(N, D, lo, hi, seed=1)
    fit = O.evaluate(obj, pop)
    f0 = fit.min()
    for g in range(60):
        s = O.step(pop, fit, 0.5, 0.9, xo, obj, lo, hi, 1, g, want_mask=True)
        m = s.mask.astype(bool)
        assert np.array_equal(s.trial[~m], pop[~m])
        assert np.all(s.fit <= fit)
        assert np.all(s.pop >= lo) and np.all(s.pop <= hi)
        assert np.array_equal(s.accept, s.ftrial < fit)
        pop, fit = s.pop, s.fit
    assert fit.min() < 0.05 * f0


def test_row_range_and_run_helper():
    N, D, obj = 20, 8, "ackley"
    pop, fit, lo, hi = _setup(N, D, obj)
    full = O.step(pop, fit, 0.5, 0.9, "nec", obj, lo, hi, 3, 1)
    part = O.step(pop, fit, 0.5, 0.9, "nec", obj, lo, hi, 3, 1, rows=(5, 11))
    assert np.array_equal(part.pop[5:11], full.pop[5:11])
    assert np.array_equal(part.pop[:5], pop[:5]) and np.array_equal(part.pop[11:], pop[11:])
    assert np.array_equal(part.draws, full.draws[5:11])
    popr, fitr, b, bf, bg, acc, sl = O.run(N, D, 0.5, 0.9, "nec", obj, lo, hi, 3, 10)
    assert fitr[b] == bf and 0 <= bg <= 10 and acc >= 0 and sl >= 10 * N
