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
            assert idx == O.argmin(fit) and f == fit[idx] and bg == 0 and np.array_equal(x, pop[idx])
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


def min_group(D):
    """Fewest lanes per row of the register kernels: ceil(ceil(D/4) / G) <= 16."""
    G = 4
    while G < 256 and -(-(-(-D // 4)) // G) > 16:
        G *= 2
    return G


def test_batch_tile_shapes_keep_draws_and_trials():
    specs = [dict(N=40, D=D, obj="rastrigin", bounds=W.BOXES["rastrigin"], xo=xo, CR=0.9, F=0.5)
             for D in (7, 100, 600, 3000) for xo in ("nec", "bin")]
    ref = None
    for mult in (1, 2, 4):
        b = DE.Batch(specs, seed=3)
        try:
            b.set_groups([min(256, min_group(sp["D"]) * mult) for sp in specs])
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
        b.prepare_run(4)                       # builds the graph only
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
            assert idx == O.argmin(fb) and f == fb[idx] and np.array_equal(x, pb[idx])
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


def test_batch_group_choice_is_bit_invariant():
    """For rows of at most one warp (register tiles of G = 4 .. 32 lanes, the
    staged kernel, or the streaming kernel) the fitness is summed in one order
    whatever the kernel, so every valid choice gives the same fitness bits,
    selections and trajectories."""
    specs = []
    k = 0
    for D in (1, 3, 10, 64, 130, 257, 600, 1000, 2000):
        for xo in ("nec", "bin", "exp"):
            obj = OBJS[k % len(OBJS)]
            specs.append(dict(N=37 + 3 * k, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=0.9, F=0.5))
            k += 1
    ref = None
    for G in (0, -4, -8, -16, -32, 4, 8, 16, 32, 2):
        b = DE.Batch(specs, seed=11)
        try:
            if G <= 0 or G == 2:   # the staged kernel with -G lanes per row, or the streaming kernel (exp / NEC)
                b.set_groups([G if sp["xo"] != "bin" else 0 for sp in specs])
            else:
                b.set_groups([max(min_group(sp["D"]), G) for sp in specs])
            for k in range(len(specs)):
                b.set_population(k, W.population(specs[k]["N"], specs[k]["D"], *specs[k]["bounds"], 70 + k))
            b.run(5)
            out = [b.population(k) for k in range(len(specs))]
            if ref is None:
                ref = out
            for k, ((p, f), (p0, f0)) in enumerate(zip(out, ref)):
                assert np.array_equal(f.view(np.uint32), f0.view(np.uint32)), (G, k)
                assert np.array_equal(p.view(np.uint32), p0.view(np.uint32)), (G, k)
        finally:
            b.close()


def test_batch_groups_validation_and_defaults():
    specs = [dict(N=20, D=D, obj="sphere", bounds=W.BOXES["sphere"], xo=xo, CR=0.9, F=0.5)
             for (D, xo) in [(10, "nec"), (2000, "exp"), (2049, "nec"), (300, "bin"), (5000, "bin")]]
    b = DE.Batch(specs, seed=1)
    default = [-32, -32, min_group(2049), min_group(300), min_group(5000)]
    try:
        assert b.groups() == default
        for bad in ([1, 1, 1, 0, 0], [0, 0, 0, 1, 0], [0, 0, 0, 2, 0], [0, 0, 0, 0, 2], [0, 0, 0, 12, 0],
                    [0, 4, 0, 0, 0], [-2, 0, 0, 0, 0], [-64, 0, 0, 0, 0], [0, 0, -32, 0, 0], [0, 0, 0, -8, 0]):
            with pytest.raises(DE.DEError):
                b.set_groups(bad)
            assert b.groups() == default
        b.set_groups([4, 32, 0, 32, 0])
        assert b.groups() == [4, 32, min_group(2049), 32, min_group(5000)]
        b.set_groups([-8, -16, 0, 0, 0])
        assert b.groups() == [-8, -16, min_group(2049), min_group(300), min_group(5000)]
        b.set_groups([1, 1, 0, 0, 0])           # the staged kernel with its default lanes
        assert b.groups() == default
        b.set_groups([2, 2, 2, 0, 0])           # the streaming kernel: exp / NEC rows of any D
        assert b.groups() == [2, 2, 2, min_group(300), min_group(5000)]
        b.set_groups([0, 0, 0, 0, 0])
        assert b.groups() == default
    finally:
        b.close()


def test_batch_autotune_keeps_state_and_results():
    """The autotuner's trial generations leave populations, fitness, counters
    and the generation as they were, and the tuned batch follows the same
    trajectory as an untuned one."""
    specs = mixed_specs()
    n = len(specs)
    a = DE.Batch(specs, seed=21)
    b = DE.Batch(specs, seed=21)
    try:
        a.run(3)
        b.run(3)
        before = [a.population(k) for k in range(n)]
        st = [a.stats(k) for k in range(n)]
        groups = a.autotune(reps=2)
        assert groups == a.groups()
        for k in range(n):
            p, f = a.population(k)
            assert np.array_equal(p.view(np.uint32), before[k][0].view(np.uint32)), k
            assert np.array_equal(f.view(np.uint32), before[k][1].view(np.uint32)), k
            assert a.stats(k) == st[k], k
        a.run(4)
        b.run(4)
        for k in range(n):
            pa, fa = a.population(k)
            pb, fb = b.population(k)
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32)), k
            assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32)), k
        assert a.stats() == b.stats()
    finally:
        a.close()
        b.close()


def test_batch_one_launch_generation_matches_the_three_launch_path():
    """A batch whose instances are all on the staged kernel runs each
    generation as one cooperative launch (plans, grid barrier, rows, close).
    Moving one instance to the register kernel switches the batch to the
    plan / rows / close launches; both paths sum fitness in one order, so the
    trajectories are bit-identical, and the one-launch path matches the
    oracle for a generation."""
    specs = []
    for k, (D, xo) in enumerate([(10, "nec"), (100, "exp"), (600, "nec"), (2000, "nec"), (33, "exp"), (1024, "nec")]):
        obj = OBJS[k % 4]
        specs.append(dict(N=50 + 7 * k, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=0.9, F=0.5))
    a = DE.Batch(specs, seed=9)
    b = DE.Batch(specs, seed=9)
    try:
        assert all(g < 0 for g in a.groups())            # every instance staged: one launch per generation
        b.set_groups([min_group(specs[0]["D"])] + [0] * (len(specs) - 1))
        a.run(6)
        b.run(6)
        for k in range(len(specs)):
            pa, fa = a.population(k)
            pb, fb = b.population(k)
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32)), k
            assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32)), k
            assert a.stats(k) == b.stats(k), k
        for k in (0, 3, 4):
            check_instance_step(a, k, specs[k], 9)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("CR", [0.0, 1.0, 0.99])
def test_batch_staged_edge_cases(CR):
    """Staged-kernel edge cases against the oracle, one generation each: Cr = 0
    (L = 1) and Cr = 1 (L = D), Cr = 0.99 (segments longer than the shared
    donor area read their donors from global memory), the minimum N = 4, and
    rows of exactly 512 float4 slots (D = 2048: one row per pass) next to
    D = 2049 (over the limit: register tiles in the same batch)."""
    specs = []
    for k, (N, D, xo) in enumerate([(4, 2048, "nec"), (9, 2047, "exp"), (40, 3, "nec"), (23, 2049, "nec"),
                                    (64, 777, "exp"), (5, 1, "nec")]):
        obj = OBJS[k % 4]
        specs.append(dict(N=N, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=CR, F=0.7))
    b = DE.Batch(specs, seed=13)
    try:
        g = b.groups()
        assert g[3] > 0 and all(v < 0 for i, v in enumerate(g) if i != 3)
        b.run(2)
        for k in range(len(specs)):
            check_instance_step(b, k, specs[k], 13)
        # the same batch with every instance staged except the one that cannot be
        only_staged = [s for s in specs if s["D"] <= 2048]
        c = DE.Batch(only_staged, seed=13)
        try:
            for k in range(len(only_staged)):
                check_instance_step(c, k, only_staged[k], 13)
        finally:
            c.close()
    finally:
        b.close()


FLOW = 2                                  # the streaming row kernel's group value


@pytest.mark.parametrize("CR", [0.9, 0.0, 1.0, 0.99])
def test_batch_streaming_kernel_matches_oracle(CR):
    """The streaming row kernel (one warp per row, chunks of 512 genes) on
    every instance: one cooperative launch per generation, each instance's
    generation against the oracle. Rows of one chunk and of several (D = 513, 1025,
    2049, 5000 and 10000: the trial of an accepted row is re-read and stored
    chunk by chunk), segments that wrap, Cr = 0 (L = 1), Cr = 1 (L = D) and
    Cr = 0.99 (segments of more than 32 slots take the per-slot path), the
    minimum N = 4, every objective."""
    specs = []
    for k, (N, D, xo) in enumerate([(4, 1, "nec"), (9, 3, "exp"), (40, 10, "nec"), (23, 129, "exp"),
                                    (64, 1024, "nec"), (17, 1025, "nec"), (8, 513, "exp"), (6, 2049, "exp"), (5, 5000, "nec"),
                                    (4, 10000, "nec"), (33, 777, "exp"), (12, 4097, "nec"), (50, 64, "nec")]):
        obj = OBJS[k % len(OBJS)]
        specs.append(dict(N=N, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=CR, F=0.6))
    b = DE.Batch(specs, seed=17)
    try:
        b.set_groups([FLOW] * len(specs))
        assert b.groups() == [FLOW] * len(specs)
        b.run(2)
        for k in range(len(specs)):
            check_instance_step(b, k, specs[k], 17)
    finally:
        b.close()


def test_batch_streaming_one_launch_matches_multi_launch_and_staged():
    """Every instance on the streaming kernel runs a generation as one
    cooperative launch; moving one instance to register tiles switches the
    batch to plan / rows / close launches, and the staged kernel sums in the
    same order: all three trajectories are bit-identical."""
    specs = []
    for k, (D, xo) in enumerate([(10, "nec"), (100, "exp"), (600, "nec"), (2000, "nec"), (33, "exp"),
                                 (1024, "nec"), (1500, "exp")]):
        obj = OBJS[k % 4]
        specs.append(dict(N=60 + 7 * k, D=D, obj=obj, bounds=W.BOXES[obj], xo=xo, CR=0.9, F=0.5))
    runs = []
    for mode in ("flow_fused", "flow_multi", "staged"):
        b = DE.Batch(specs, seed=19)
        try:
            if mode == "flow_fused":
                b.set_groups([FLOW] * len(specs))
            elif mode == "flow_multi":
                b.set_groups([min_group(specs[0]["D"])] + [FLOW] * (len(specs) - 1))
            b.run(7)
            runs.append([(b.population(k), b.stats(k)) for k in range(len(specs))])
        finally:
            b.close()
    for k in range(len(specs)):
        (p0, f0), s0 = runs[0][k]
        for r in runs[1:]:
            (p1, f1), s1 = r[k]
            assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32)), k
            assert np.array_equal(f0.view(np.uint32), f1.view(np.uint32)), k
            assert s0 == s1, k


def test_batch_streaming_evaluation_matches_oracle():
    """Parent evaluation (set_population without fitness) on the streaming
    kernel: the FP32 fitness of every row within tolerance of the oracle."""
    specs = [dict(N=30 + k, D=D, obj=OBJS[k % len(OBJS)], bounds=W.BOXES[OBJS[k % len(OBJS)]], xo="nec", CR=0.9,
                  F=0.5) for k, D in enumerate([1, 7, 300, 1024, 1030, 3333])]
    b = DE.Batch(specs, seed=23)
    try:
        b.set_groups([FLOW] * len(specs))
        for k, s in enumerate(specs):
            pop = W.population(s["N"], s["D"], *s["bounds"], 300 + k)
            b.set_population(k, pop)
            _, f = b.population(k)
            f64 = O.evaluate(s["obj"], pop)
            assert np.all(np.abs(f - f64) <= tol(f64)), k
            x, fb, idx, _ = b.best(k)
            assert idx == O.argmin(f) and fb == f[idx]
    finally:
        b.close()
