"""GPU parity of the batched path (many independent instances, one launch
per generation) against the oracle, instance by instance. Instance k draws
from Philox instance field k, which the oracle takes as `inst`."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def tol(f):
    return RTOL * np.maximum(1.0, np.abs(f))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    DE.load_library()


OBJS = ["sphere", "rastrigin", "ackley", "rosenbrock", "griewank", "elliptic"]


def mixed_specs():
    specs = []
    shapes = [(4, 1), (37, 10), (64, 29), (100, 130), (20, 1000), (50, 2000), (9, 4097), (300, 64), (16, 257)]
    k = 0
    for (N, D) in shapes:
        for xo, CR in (("nec", 0.9), ("bin", 0.5), ("exp", 0.7)):
            obj = OBJS[k % len(OBJS)]
            specs.append(dict(N=N, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=CR, F=0.5 + 0.05 * (k % 3)))
            k += 1
    return specs


def check_instance_step(b, k, spec, seed, pop=None):
    N, D, obj, xo, CR, F = spec["N"], spec["D"], spec["obj"], spec["xo"], spec["CR"], spec["F"]
    lo, hi = spec["bounds"]
    if pop is None:
        pop = W.population(N, D, lo, hi, 1000 + k)
    b.set_population(k, pop)
    gp, gfit = b.population(k)
    assert np.array_equal(gp.view(np.uint32), pop.view(np.uint32))
    fit64 = O.evaluate(obj, pop)
    assert np.all(np.abs(gfit - fit64) <= tol(fit64)), "instance %d parent fitness" % k
    g = b.stats(k)["generation"]
    trial, ft, acc, draws = b.debug_step(k)
    s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, inst=k)
    assert np.array_equal(draws, s.draws), "instance %d draws" % k
    assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32)), "instance %d trials" % k
    assert np.all(np.abs(ft - s.ftrial) <= tol(s.ftrial)), "instance %d trial fitness" % k
    amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
    assert np.array_equal(acc[~amb], s.accept[~amb]), "instance %d selection" % k
    np_, nf = b.population(k)
    assert np.array_equal(np_.view(np.uint32), np.where(acc[:, None], trial, pop).view(np.uint32))


def test_batch_init_parity():
    specs = mixed_specs()
    b = DE.Batch(specs, seed=5)
    try:
        assert len(b) == len(specs) and DE.de_batch_size(b.ctx) == len(specs)
        for k, sp in enumerate(specs):
            lo, hi = sp["bounds"]
            pop, fit = b.population(k)
            ref = O.init(sp["N"], sp["D"], lo, hi, 5, inst=k)
            assert np.array_equal(pop.view(np.uint32), ref.view(np.uint32)), k
            f64 = O.evaluate(sp["obj"], ref)
            assert np.all(np.abs(fit - f64) <= tol(f64)), k
            x, f, idx, bg = b.best(k)
            assert idx == int(np.argmin(fit)) and f == fit[idx] and bg == 0 and np.array_equal(x, pop[idx])
    finally:
        b.close()


def test_batch_one_generation_parity_every_instance():
    specs = mixed_specs()
    b = DE.Batch(specs, seed=9)
    try:
        for k, sp in enumerate(specs):
            check_instance_step(b, k, sp, 9)
    finally:
        b.close()


def test_batch_tile_shapes_keep_draws_and_trials():
    specs = [dict(N=40, D=D, obj="rastrigin", bounds=W.BOXES["rastrigin"], xo=xo, CR=0.9, F=0.5)
             for D in (7, 100, 600) for xo in ("nec", "bin")]
    ref = None
    for mult in (1, 2, 4):
        b = DE.Batch(specs, seed=3)
        try:
            b.set_groups([min(256, g * mult) for g in b.groups()])
            out = []
            for k, sp in enumerate(specs):
                # a fresh population right before its step: the trial depends only on it and the generation
                b.set_population(k, W.population(sp["N"], sp["D"], -5.12, 5.12, 50 + k))
                out.append(b.debug_step(k))
            if ref is None:
                ref = out
            for (t, f, a, d), (t0, f0, a0, d0) in zip(out, ref):
                assert np.array_equal(d, d0)
                assert np.array_equal(t.view(np.uint32), t0.view(np.uint32))
                assert np.allclose(f, f0, rtol=2 * RTOL, atol=2 * RTOL)
        finally:
            b.close()


def test_batch_run_graph_stats_and_best():
    specs = mixed_specs()[:12]
    a = DE.Batch(specs, seed=4)
    b = DE.Batch(specs, seed=4)
    try:
        for _ in range(7):
            a.step()
        b.run(3)
        b.run(4)
        tot_acc = tot_msk = 0
        best = np.inf
        for k, sp in enumerate(specs):
            pa, fa = a.population(k)
            pb, fb = b.population(k)
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
            assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
            sk = b.stats(k)
            assert sk == a.stats(k) and sk["generation"] == 7
            tot_acc += sk["accepts"]
            tot_msk += sk["masked_genes"]
            x, f, idx, bg = b.best(k)
            assert idx == int(np.argmin(fb)) and f == fb[idx] and np.array_equal(x, pb[idx])
            assert f <= sk["best_f"] + 0.0 and 0 <= bg <= 7
            best = min(best, f)
        st = b.stats()
        assert st["generation"] == 7 and st["accepts"] == tot_acc and st["masked_genes"] == tot_msk
        assert st["best_f"] == best
    finally:
        a.close()
        b.close()


def test_batch_rejects_single_population_calls():
    b = DE.Batch([dict(N=8, D=4, obj="sphere", bounds=(-1.0, 1.0))], seed=1)
    try:
        with pytest.raises(DE.DEError) as e:
            DE.de_best(b.ctx)
        assert e.value.code == DE.DE_ESTATE
        with pytest.raises(DE.DEError) as e:
            DE.de_save(b.ctx)
        assert e.value.code == DE.DE_EUNSUPPORTED
    finally:
        b.close()


def test_batched_512_instance_workload_sampled():
    """The 512-instance workload (D log-uniform in [10, 2000], N = min(10 D,
    4096), objectives round-robin, NEC, F = 0.5, Cr = 0.9): every instance
    advances; sampled instances match the oracle one generation exactly."""
    specs = [dict(N=s.N, D=s.D, obj=s.objective, bounds=W.BOXES[s.objective], xo="nec", CR=0.9, F=0.5)
             for s in W.batched_specs()]
    b = DE.Batch(specs, seed=4)
    try:
        b.run(3)
        st = b.stats()
        assert st["generation"] == 3
        sizes = np.array([s["N"] * s["D"] for s in specs])
        picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), 7, 300]
        for k in picks:
            check_instance_step(b, k, specs[k], 4)
        assert b.stats()["generation"] == 3 + len(picks)
    finally:
        b.close()
