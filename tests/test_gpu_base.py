"""GPU parity of the base index rules (Alg. 3-6 and DE/best/1) against the
oracle: draws (base and difference rows, j_rand, L) and trials bit-exact,
fitness within tolerance, selections identical outside the ambiguity band,
in every generation kernel, the batched path and the rotated path."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5
BASES = ["random", "offset", "permutation", "best"]


def tol(f):
    return RTOL * np.maximum(1.0, np.abs(f))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    DE.load_library()


def step_parity(opt, pop, obj, xo, F, CR, lo, hi, seed, base, **okw):
    opt.set_population(pop)
    _, gfit = opt.population()
    fit64 = O.evaluate(obj, pop, **okw)
    st = opt.stats()
    g, best = st["generation"], st["best_index"]        # the best row the generation starts from
    trial, ft, acc, draws = opt.debug_step()
    s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, base=base, best=best, **okw)
    assert np.array_equal(draws, s.draws), "draws"
    assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32)), "trials"
    assert np.all(np.abs(ft - s.ftrial) <= tol(s.ftrial)), "trial fitness"
    amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
    assert np.array_equal(acc[~amb], s.accept[~amb]), "selection"
    if base == "best":
        assert np.all(draws[:, 0] == best)
    return s


@pytest.mark.parametrize("base", BASES)
@pytest.mark.parametrize("xo,kernel", [("bin", 1), ("exp", 1), ("nec", 1), ("bin", 3), ("nec", 3), ("exp", 2),
                                       ("nec", 2)])
@pytest.mark.parametrize("N,D", [(37, 29), (300, 2500)])
def test_base_rules_one_generation(base, xo, kernel, N, D):
    obj, F, CR, seed = "rastrigin", 0.6, 0.9, 21
    lo, hi = W.BOXES[obj]
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=(lo, hi), seed=seed)
    try:
        if kernel == 2 and opt.kernel() != 2:
            opt.set_kernel(2)
        elif kernel != 2:
            opt.set_kernel(kernel)
        opt.set_base(base)
        assert opt.base() == base
        step_parity(opt, W.population(N, D, lo, hi, 5), obj, xo, F, CR, lo, hi, seed, base)
    finally:
        opt.close()


@pytest.mark.parametrize("base", BASES)
def test_base_rules_lockstep_generations(base):
    """40 generations of Rosenbrock, every generation checked against the
    oracle stepping from the GPU's own population (best row included)."""
    N, D, F, CR, seed, obj, xo = 100, 50, 0.65, 0.95, 1, "rosenbrock", "bin"
    lo, hi = W.BOXES[obj]
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=(lo, hi), seed=seed)
    try:
        opt.set_base(base)
        for _ in range(40):
            pop, _ = opt.population()
            fit64 = O.evaluate(obj, pop)
            st = opt.stats()
            g, best = st["generation"], st["best_index"]
            trial, ft, acc, draws = opt.debug_step()
            s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, base=base, best=best)
            assert np.array_equal(draws, s.draws)
            assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32))
            amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
            assert np.array_equal(acc[~amb], s.accept[~amb])
    finally:
        opt.close()


def test_base_rule_graph_run_matches_steps():
    """de_run (graph replay) under a base rule equals stepping one by one."""
    N, D, obj = 64, 300, "ackley"
    a = DE.Optimizer(N, D, F=0.5, CR=0.9, xo="nec", obj=obj, bounds=W.BOXES[obj], seed=3)
    b = DE.Optimizer(N, D, F=0.5, CR=0.9, xo="nec", obj=obj, bounds=W.BOXES[obj], seed=3)
    try:
        a.set_base("permutation")
        b.set_base("permutation")
        a.run(12)
        for _ in range(12):
            b.step()
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert a.stats() == b.stats()
    finally:
        a.close()
        b.close()


def test_base_rules_batched():
    specs = [dict(N=N, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=0.9, F=0.5)
             for (N, D, obj, xo) in [(40, 30, "sphere", "nec"), (60, 600, "rastrigin", "bin"),
                                     (20, 2100, "ackley", "exp")]]
    for base in BASES:
        bt = DE.Batch(specs, seed=7)
        try:
            bt.set_base(base)
            for k, sp in enumerate(specs):
                lo, hi = sp["bounds"]
                pop = W.population(sp["N"], sp["D"], lo, hi, 40 + k)
                bt.set_population(k, pop)
                fit64 = O.evaluate(sp["obj"], pop)
                st = bt.stats(k)
                g, best = st["generation"], O.argmin(bt.population(k)[1])
                trial, ft, acc, draws = bt.debug_step(k)
                s = O.step(pop, fit64, sp["F"], sp["CR"], sp["xo"], sp["obj"], lo, hi, 7, g, inst=k, base=base,
                           best=best)
                assert np.array_equal(draws, s.draws), (base, k)
                assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32)), (base, k)
        finally:
            bt.close()


def test_base_best_rotated():
    """The shifted-rotated path draws through the same rule."""
    N, D, obj = 64, 128, "sr_rastrigin"
    o = W.shift_vector(D, seed=2)
    R = W.rotation(D, seed=3)
    lo, hi = W.BOXES[obj]
    opt = DE.Optimizer(N, D, F=0.5, CR=0.9, xo="nec", obj=obj, bounds=(lo, hi), seed=4,
                       params={"shift": o, "rotation": R, "prec": "fp32"})
    try:
        opt.set_base("best")
        step_parity(opt, W.population(N, D, lo, hi, 8), obj, "nec", 0.5, 0.9, lo, hi, 4, "best", shift=o, rot=R)
    finally:
        opt.close()
