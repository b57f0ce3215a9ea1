"""Parity at the benchmark's full size (N = 16384, D = 10000), in the launch
configuration bench.py times (the automatically selected kernel and shape).

The oracle recomputes sampled rows one by one (draws, trial, FP64 fitness,
decision) from the same seeded population; every row is checked against
properties that hold at any size (unmasked genes are the parent's, the
masked genes form the circular segment of length L from j_rand, genes stay
in the box, the decision matches the GPU's own FP32 fitness values)."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, D, F, CR = 16384, 10000, 0.5, 0.9
SAMPLES = ((0, 24), (8181, 8205), (16360, 16384))


def tol(f):
    return 1e-5 * np.maximum(1.0, np.abs(f))


@pytest.fixture(scope="module")
def population():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return {obj: W.population(N, D, *W.BOXES[obj], seed=123) for obj in ("rosenbrock", "ackley")}


@pytest.mark.parametrize("xo,obj", [("nec", "rosenbrock"), ("exp", "rosenbrock"), ("nec", "ackley"),
                                    ("bin", "rosenbrock")])
def test_full_size_sampled_parity(population, xo, obj):
    lo, hi = W.BOXES[obj]
    pop = population[obj]
    seed = 1
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=(lo, hi), seed=seed)
    try:
        assert opt.kernel() == (3 if xo == "bin" else 2)     # the kernels bench.py times at this size
        opt.set_population(pop)
        _, fit32 = opt.population()
        opt.run(2)                                       # the timed state: a few generations in
        pop_g, fit_g = opt.population()
        g = opt.stats()["generation"]
        trial, ft, acc, draws = opt.debug_step()

        # properties of every row
        jr, L = draws[:, 3].astype(np.int64), draws[:, 4].astype(np.int64)
        assert np.all((draws[:, :3] >= 0) & (draws[:, :3] < N))
        assert np.all(draws[:, 0] != np.arange(N)) and np.all(draws[:, 1] != draws[:, 0])
        assert np.all(draws[:, 2] != draws[:, 1]) and np.all(draws[:, 2] != draws[:, 0])
        assert np.all((trial >= lo) & (trial <= hi))
        assert np.array_equal(acc, ft < fit_g)
        if xo != "bin":
            assert np.all((L >= 1) & (L <= D))
            for i in range(0, N, 97):
                seg = ((np.arange(D) - jr[i]) % D) < L[i]
                assert np.array_equal(trial[i, ~seg], pop_g[i, ~seg])
        else:
            changed = trial != pop_g
            assert np.all(changed.sum(1) <= L)

        # sampled rows against the oracle (same population, same generation)
        for (i0, i1) in SAMPLES:
            fit64 = np.full(N, np.inf)
            fit64[i0:i1] = O.evaluate(obj, pop_g[i0:i1])
            s = O.step(pop_g, fit64, F, CR, xo, obj, lo, hi, seed, g, rows=(i0, i1))
            assert np.array_equal(draws[i0:i1], s.draws)
            assert np.array_equal(trial[i0:i1].view(np.uint32), s.trial.view(np.uint32))
            assert np.all(np.abs(ft[i0:i1] - s.ftrial) <= tol(s.ftrial))
            assert np.all(np.abs(fit_g[i0:i1] - fit64[i0:i1]) <= tol(fit64[i0:i1]))
            amb = np.abs(s.ftrial - fit64[i0:i1]) <= tol(s.ftrial) + tol(fit64[i0:i1])
            assert np.array_equal(acc[i0:i1][~amb], s.accept[~amb])
    finally:
        opt.close()
