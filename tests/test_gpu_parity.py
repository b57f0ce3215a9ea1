"""GPU parity of the fused generation kernel against the CPU oracle.

Every test here runs libde.so's CUDA kernels through the C ABI (ctypes
binding) and compares element by element with the oracle on the same seeded
inputs:
  - draws (r1, r2, r3, j_rand, L) and trial vectors: bit-exact;
  - FP32 fitness: |f32 - f64| <= 1e-5 max(1, |f64|);
  - selections: identical wherever the FP64 margin exceeds the two
    tolerances (|f(u) - f(x)| > tol(u) + tol(x)); the rest is counted.
"""
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


def make(N, D, xo, obj, CR=0.9, F=0.5, seed=1, bounds=None):
    lo, hi = bounds if bounds is not None else W.BOXES[obj]
    return DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=(lo, hi), seed=seed), lo, hi


def check_fitness(f32, f64, what):
    f32 = np.asarray(f32, np.float64)
    bad = np.abs(f32 - f64) > tol(f64)
    assert not bad.any(), "%s: %d rows off, e.g. %r vs %r" % (what, bad.sum(), f32[bad][:3], f64[bad][:3])


def one_step_parity(opt, lo, hi, xo, obj, F, CR, seed, pop=None, repair="clip"):
    """Shared parent population -> one GPU debug step and one oracle step."""
    N, D = opt.N, opt.D
    if pop is None:
        pop = W.population(N, D, lo, hi, seed + 100)
    opt.set_population(pop)
    gpu_pop, gpu_fit = opt.population()
    assert np.array_equal(gpu_pop.view(np.uint32), pop.view(np.uint32))
    fit64 = O.evaluate(obj, pop)
    check_fitness(gpu_fit, fit64, "parent fitness")
    g = opt.stats()["generation"]
    trial, ft, acc, draws = opt.debug_step()
    s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, repair=repair)
    assert np.array_equal(draws, s.draws), "draws differ"
    assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32)), "trials differ"
    check_fitness(ft, s.ftrial, "trial fitness")
    amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
    assert np.array_equal(acc[~amb], s.accept[~amb]), "selection differs outside the ambiguity band"
    new_pop, new_fit = opt.population()
    exp_pop = np.where(acc[:, None], trial, pop)
    assert np.array_equal(new_pop.view(np.uint32), exp_pop.view(np.uint32))
    assert np.array_equal(new_fit[acc], ft[acc]) and np.array_equal(new_fit[~acc], gpu_fit[~acc])
    return s, acc, int(amb.sum())


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("obj", ["sphere", "rastrigin", "ackley", "rosenbrock", "griewank", "elliptic"])
@pytest.mark.parametrize("N,D,CR", [(37, 29, 0.9), (64, 1000, 0.5), (20, 4097, 0.9), (48, 130, 0.1)])
def test_one_generation_parity(xo, obj, N, D, CR):
    F, seed = 0.5, 7
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        one_step_parity(opt, lo, hi, xo, obj, F, CR, seed)
    finally:
        opt.close()


@pytest.mark.parametrize("N,D", [(16, 8), (100, 30), (7, 1001), (5, 9999)])
def test_init_parity(N, D):
    for obj in ("rastrigin", "ackley"):
        lo, hi = W.BOXES[obj]
        opt = DE.Optimizer(N, D, 0.5, 0.9, "nec", obj, (lo, hi), seed=3)
        try:
            pop, fit = opt.population()
            ref = O.init(N, D, lo, hi, 3)
            assert np.array_equal(pop.view(np.uint32), ref.view(np.uint32))
            check_fitness(fit, O.evaluate(obj, ref), "initial fitness")
            x, f, idx, bg = opt.best()
            assert idx == O.argmin(fit) and f == fit[idx] and bg == 0
            assert np.array_equal(x, pop[idx])
        finally:
            opt.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_lockstep_generations_sphere_N100_D30(xo):
    """200 generations of the sphere workload; every generation is checked
    against the oracle stepping from the GPU's own population."""
    N, D, F, CR, seed, obj = 100, 30, 0.5, 0.9, 1, "sphere"
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        ambiguous = 0
        f_start = opt.best()[1]
        for g in range(200):
            pop, fit32 = opt.population()
            fit64 = O.evaluate(obj, pop)
            check_fitness(fit32, fit64, "gen %d fitness" % g)
            trial, ft, acc, draws = opt.debug_step()
            s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g)
            assert np.array_equal(draws, s.draws)
            assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32))
            amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
            assert np.array_equal(acc[~amb], s.accept[~amb])
            ambiguous += int((acc != s.accept).sum())
        _, f_end, _, bg = opt.best()
        assert f_end < 1e-2 * f_start and bg > 100
        print("decisions that differed inside the ambiguity band:", ambiguous)
    finally:
        opt.close()


@pytest.mark.parametrize("xo", ["bin", "nec"])
@pytest.mark.parametrize("obj,D,N,F,CR,box,b,G", [
    ("ackley", 1000, 500, 0.5, 0.2, (-30.0, 30.0), 0.02, 40),
    ("griewank", 500, 300, 0.25, 0.45, (-400.0, 400.0), 0.2, 60),
    ("rosenbrock", 50, 100, 0.65, 0.95, (-5.12, 5.12), 0.2, 300),
])
def test_lockstep_generations_paper_workloads(xo, obj, D, N, F, CR, box, b, G):
    """The paper's three DE workloads (its parameter table): every generation
    checked against the oracle stepping from the GPU's own population."""
    seed = 1
    lo, hi = box
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=box, seed=seed, params={"ackley_b": b})
    try:
        for g in range(G):
            pop, fit32 = opt.population()
            fit64 = O.evaluate(obj, pop, ackley_b=b)
            check_fitness(fit32, fit64, "gen %d fitness" % g)
            trial, ft, acc, draws = opt.debug_step()
            s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, ackley_b=b)
            assert np.array_equal(draws, s.draws)
            assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32))
            check_fitness(ft, s.ftrial, "gen %d trial fitness" % g)
            amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
            assert np.array_equal(acc[~amb], s.accept[~amb])
    finally:
        opt.close()


def test_run_graph_matches_steps_and_stats():
    N, D = 96, 200
    a, lo, hi = make(N, D, "nec", "rastrigin", seed=5)
    b, _, _ = make(N, D, "nec", "rastrigin", seed=5)
    try:
        acc_total, masked_total = 0, 0
        for _ in range(12):
            _, _, acc, draws = a.debug_step()
            acc_total += int(acc.sum())
            masked_total += int(draws[:, 4].astype(np.int64).sum())
        b.run(5)
        b.run(7)
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
        sa, sb = a.stats(), b.stats()
        assert sa["generation"] == sb["generation"] == 12
        assert sa["accepts"] == sb["accepts"] == acc_total
        assert sa["masked_genes"] == sb["masked_genes"] == masked_total
        x, f, idx, bg = b.best()
        assert idx == O.argmin(fb) and f == fb[idx] and np.array_equal(x, pb[idx])
        assert 0 <= bg <= 12 and sb["best_gen"] == bg
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_prepared_run_changes_nothing_until_launched(xo):
    """de_prepare_run captures the graph without running it: the population,
    fitness and counters stay as they were, and the prepared runs then give
    what unprepared ones give."""
    N, D = 96, 200
    a, _, _ = make(N, D, xo, "rastrigin", seed=8)
    b, _, _ = make(N, D, xo, "rastrigin", seed=8)
    try:
        p0, f0 = b.population()
        b.prepare_run(6)
        b.prepare_run(6)                       # cached: a second call builds nothing
        b.prepare_run(1)
        b.prepare_run(0)
        b.synchronize()
        p1, f1 = b.population()
        assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32))
        assert np.array_equal(f0.view(np.uint32), f1.view(np.uint32))
        assert b.stats()["generation"] == 0
        a.run(6)
        a.run(6)
        b.run(6)
        b.run(6)
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
        assert a.stats() == b.stats() and b.stats()["generation"] == 12
        with pytest.raises(DE.DEError):
            b.prepare_run(-1)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_save_load_resumes_bit_identically(xo):
    N, D = 50, 77
    a, lo, hi = make(N, D, xo, "ackley", CR=0.7, seed=9)
    b, _, _ = make(N, D, xo, "ackley", CR=0.7, seed=9)
    try:
        a.run(6)
        blob = a.save()
        a.run(9)
        b.load(blob)
        b.run(9)
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
        assert a.stats() == b.stats()
        assert a.best()[1:] == b.best()[1:]
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_edge_cases(xo):
    F = 0.5
    # D = 1: the only gene is j_rand and L = 1 = D
    for (N, D, CR, obj) in [(4, 1, 0.9, "sphere"), (4, 5, 0.0, "rastrigin"), (9, 33, 1.0, "rosenbrock"),
                            (600, 3, 0.5, "griewank"), (4, 7, 0.3, "elliptic")]:
        opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=11)
        try:
            s, acc, _ = one_step_parity(opt, lo, hi, xo, obj, F, CR, 11)
            if CR == 0.0:
                assert np.all(s.L == 1)
            if CR == 1.0 or D == 1:
                assert np.all(s.L == D)
        finally:
            opt.close()


def test_maximum_row_length_and_launch_shapes():
    N, D, obj, xo = 6, 32768, "rosenbrock", "nec"
    opt, lo, hi = make(N, D, xo, obj, CR=0.99, seed=2)
    try:
        one_step_parity(opt, lo, hi, xo, obj, 0.5, 0.99, 2)
    finally:
        opt.close()
    # the same step under other launch shapes: identical draws and trials
    N, D = 12, 1000
    pop = W.population(N, D, -5.12, 5.12, 4)
    ref = None
    for (T, V) in [(256, 1), (128, 2), (64, 4), (32, 8), (32, 16)]:
        opt, lo, hi = make(N, D, "bin", "rastrigin", CR=0.5, seed=4)
        try:
            opt.set_launch(T, V)
            assert opt.launch() == (T, V)
            opt.set_population(pop)
            trial, ft, acc, draws = opt.debug_step()
            if ref is None:
                ref = (trial, ft, draws)
            assert np.array_equal(trial.view(np.uint32), ref[0].view(np.uint32))
            assert np.array_equal(draws, ref[2])
            assert np.allclose(ft, ref[1], rtol=RTOL, atol=RTOL)
        finally:
            opt.close()


def test_ties_keep_parent_on_gpu():
    N, D = 8, 10
    pop = np.tile(W.population(1, D, -5, 5, 3), (N, 1))
    opt, lo, hi = make(N, D, "nec", "rastrigin", seed=1)
    try:
        opt.set_population(pop)
        trial, ft, acc, _ = opt.debug_step()
        assert np.array_equal(trial, pop) and not acc.any()
    finally:
        opt.close()


# ---- the pipelined kernel (exp / NEC) --------------------------------------------------------
@pytest.mark.parametrize("xo", ["exp", "nec"])
@pytest.mark.parametrize("obj", ["sphere", "rastrigin", "ackley", "rosenbrock", "griewank", "elliptic"])
@pytest.mark.parametrize("N,D,CR", [(37, 29, 0.9), (300, 1000, 0.5), (20, 4097, 0.9), (160, 2048, 0.1)])
def test_pipeline_kernel_parity(xo, obj, N, D, CR):
    F, seed = 0.5, 13
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        opt.set_kernel(2)
        assert opt.kernel() == 2
        one_step_parity(opt, lo, hi, xo, obj, F, CR, seed)
    finally:
        opt.close()


@pytest.mark.parametrize("xo", ["exp", "nec"])
@pytest.mark.parametrize("N,D,CR,consumers,stages", [
    (64, 4000, 0.999, 256, 0),     # long segments: many exceed the donor span buffer (global fallback)
    (40, 8000, 0.9999, 128, 3),    # NEC table larger than the shared-memory copy (global search)
    (4, 1, 0.9, 32, 0),            # D = 1
    (500, 3, 0.0, 512, 2),         # Cr = 0: L = 1
    (33, 130, 1.0, 64, 5),         # Cr = 1: L = D, the segment wraps onto itself
    (2000, 5000, 0.9, 128, -2),    # two CTAs per SM (stages as many as fit)
])
def test_pipeline_kernel_edges(xo, N, D, CR, consumers, stages):
    F, seed, obj = 0.7, 21, "rosenbrock"
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        opt.set_kernel(2)
        cps = 2 if stages < 0 else 1
        stages = max(stages, 0)
        opt.set_pipeline(consumers, stages, cps)
        nc, st, span, cps = opt.pipeline()
        assert nc == consumers and (stages == 0 or st == stages) and span >= 16
        s, acc, _ = one_step_parity(opt, lo, hi, xo, obj, F, CR, seed)
        if CR == 0.0:
            assert np.all(s.L == 1)
        if CR == 1.0:
            assert np.all(s.L == D)
    finally:
        opt.close()


@pytest.mark.parametrize("xo", ["exp", "nec"])
def test_pipeline_matches_row_kernel_over_generations(xo):
    N, D, obj = 700, 2500, "ackley"
    a, lo, hi = make(N, D, xo, obj, CR=0.9, seed=3)
    b, _, _ = make(N, D, xo, obj, CR=0.9, seed=3)
    try:
        a.set_kernel(1)
        b.set_kernel(2)
        for g in range(6):
            ta, fa, acca, da = a.debug_step()
            tb, fb, accb, db = b.debug_step()
            assert np.array_equal(da, db)
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.allclose(fa, fb, rtol=2 * RTOL, atol=2 * RTOL)
            # the two kernels reduce in different orders: decisions may differ only in near-ties
            pa, ffa = a.population()
            pb, ffb = b.population()
            if not np.array_equal(pa.view(np.uint32), pb.view(np.uint32)):
                b.set_population(pa, ffa)       # re-align and continue
        b.run(4)
        st = b.stats()
        assert st["generation"] == 10
    finally:
        a.close()
        b.close()


def test_pipeline_graph_save_load():
    N, D, xo, obj = 300, 3000, "nec", "rastrigin"
    a, lo, hi = make(N, D, xo, obj, CR=0.9, seed=8)
    b, _, _ = make(N, D, xo, obj, CR=0.9, seed=8)
    try:
        assert a.kernel() == 2 and b.kernel() == 2            # chosen automatically at D >= 2048
        a.run(5)
        blob = a.save()
        a.run(7)
        b.load(blob)
        for _ in range(7):
            b.step()
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
        assert a.stats() == b.stats()
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("D", [2048, 10000, 16000])
def test_automatic_kernel_choice_at_large_rows(D):
    for xo in ("exp", "nec", "bin"):
        opt, lo, hi = make(64, D, xo, "rosenbrock", seed=1)
        try:
            assert opt.kernel() == (3 if xo == "bin" else 2)
            if xo != "bin":
                nc, stages, span, cps = opt.pipeline()
                assert stages >= 2 and cps in (1, 2) and nc == 256
        finally:
            opt.close()


# ---- the streaming kernel (one warp per row, chunks of 512 genes) ----------------------------
@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("obj", ["sphere", "rastrigin", "ackley", "rosenbrock", "griewank", "elliptic"])
@pytest.mark.parametrize("N,D,CR", [(37, 29, 0.9), (64, 1000, 0.5), (20, 4097, 0.9), (48, 513, 0.1),
                                    (9, 9999, 0.9)])
def test_stream_kernel_parity(xo, obj, N, D, CR):
    F, seed = 0.5, 17
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        opt.set_kernel(3)
        assert opt.kernel() == 3
        one_step_parity(opt, lo, hi, xo, obj, F, CR, seed)
    finally:
        opt.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("N,D,CR", [(4, 1, 0.9), (500, 3, 0.0), (33, 130, 1.0), (17, 2048, 0.9)])
def test_stream_kernel_edges(xo, N, D, CR):
    F, seed, obj = 0.7, 23, "rosenbrock"
    opt, lo, hi = make(N, D, xo, obj, CR=CR, F=F, seed=seed)
    try:
        opt.set_kernel(3)
        s, acc, _ = one_step_parity(opt, lo, hi, xo, obj, F, CR, seed)
        if xo != "bin" and CR == 0.0:
            assert np.all(s.L == 1)
        if CR == 1.0:
            assert np.all(s.L == D)                # every gene crosses (binomial: the mask popcount)
    finally:
        opt.close()


def test_stream_matches_row_kernel_over_generations():
    """Binomial, Ackley, 8 generations: the two kernels draw, cross and mutate
    identically; their FP32 sums differ only in order."""
    N, D, obj = 600, 3000, "ackley"
    a, lo, hi = make(N, D, "bin", obj, CR=0.9, seed=4)
    b, _, _ = make(N, D, "bin", obj, CR=0.9, seed=4)
    try:
        a.set_kernel(1)
        assert b.kernel() == 3                     # chosen automatically for binomial at D >= 2048
        for g in range(8):
            ta, fa, acca, da = a.debug_step()
            tb, fb, accb, db = b.debug_step()
            assert np.array_equal(da, db)
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.allclose(fa, fb, rtol=2 * RTOL, atol=2 * RTOL)
            pa, ffa = a.population()
            pb, ffb = b.population()
            if not np.array_equal(pa.view(np.uint32), pb.view(np.uint32)):
                b.set_population(pa, ffa)
        b.run(5)
        st = b.stats()
        assert st["generation"] == 13
        pop, fit = b.population()
        assert np.all(np.abs(fit - O.evaluate(obj, pop)) <= tol(O.evaluate(obj, pop)))
    finally:
        a.close()
        b.close()


def test_best_async_record_matches_best():
    """de_best_async queues the same best row and value that de_best returns."""
    N, D = 64, 37
    opt = DE.Optimizer(N, D, F=0.5, CR=0.9, xo="nec", obj="rastrigin", bounds=W.BOXES["rastrigin"], seed=3)
    try:
        import torch
        rec = DE.best_record_bytes(D)
        ring = torch.empty(3 * rec, dtype=torch.uint8).pin_memory().numpy()
        for k in range(3):
            opt.step()
            DE.de_best_async(opt.ctx, ring[k * rec:(k + 1) * rec], D)
        DE.de_synchronize(opt.ctx)
        f, idx, gen, x = DE.parse_best_record(ring[2 * rec:], D)
        x2 = np.empty(D, dtype=np.float32)
        f2, idx2, gen2 = DE.de_best(opt.ctx, x2)
        assert (f, idx, gen) == (f2, idx2, gen2)
        assert np.array_equal(x.view(np.uint32), x2.view(np.uint32))
        fs = [DE.parse_best_record(ring[k * rec:(k + 1) * rec], D)[0] for k in range(3)]
        assert fs[0] >= fs[1] >= fs[2]
    finally:
        opt.close()


@pytest.mark.parametrize("kernel", [1, 3])
@pytest.mark.parametrize("CR", [1.0 - 2.0**-40, 2.0**-33, 0.5, 1.0 - 2.0**-32])
def test_binomial_threshold_extremes(kernel, CR):
    """The binomial test w < ceil(Cr 2^32) at the ends of its range, on the
    row-per-CTA kernel (1) and the streaming kernel (3): Cr within 2^-32 of
    1 makes the threshold 2^32 (every word passes, the 32-bit comparison
    cannot say so), Cr = 2^-33 makes it 1 (only the word 0 passes), Cr = 0.5
    is a power of two. Masks, trials and selections against the oracle."""
    F, seed, obj = 0.6, 29, "sphere"
    for (N, D) in ((40, 130), (9, 1001)):
        opt, lo, hi = make(N, D, "bin", obj, CR=CR, F=F, seed=seed)
        try:
            opt.set_kernel(kernel)
            s, acc, _ = one_step_parity(opt, lo, hi, "bin", obj, F, CR, seed)
            if CR > 1.0 - 2.0**-32:
                assert np.all(s.L == D)
            if CR < 2.0**-32:
                assert np.all(s.L <= 2)                # j_rand, and a word 0 with probability 2^-32 per gene
        finally:
            opt.close()


@pytest.mark.parametrize("xo,kernel", [("bin", 1), ("exp", 1), ("nec", 1), ("exp", 2), ("nec", 2), ("bin", 3),
                                       ("nec", 3)])
def test_midpoint_repair_parity(xo, kernel):
    """DE_REPAIR_MIDPOINT: a mutant gene outside the box becomes the midpoint
    of the violated bound and the target gene, in each kernel (row per CTA,
    pipelined, streaming), bit for bit with the oracle; F = 0.9 puts many
    mutants outside the box."""
    F, CR, seed, obj = 0.9, 0.9, 31, "rastrigin"
    for (N, D) in ((40, 130), (12, 4100)):
        if kernel == 2 and D < 2048:
            continue                                    # the pipelined kernel is for long rows
        lo, hi = W.BOXES[obj]
        opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=(lo, hi), seed=seed,
                           params={"repair": "midpoint"})
        try:
            opt.set_kernel(kernel)
            s, acc, _ = one_step_parity(opt, lo, hi, xo, obj, F, CR, seed, repair="midpoint")
            c = O.step(W.population(N, D, lo, hi, seed + 100), np.full(N, np.inf), F, CR, xo, obj, lo, hi, seed,
                       0, repair="clip")
            assert not np.array_equal(s.trial, c.trial)  # some genes were repaired differently from clipping
        finally:
            opt.close()


def test_repair_mode_in_checkpoints():
    """A checkpoint records the repair mode; loading it into a context with the
    other mode is refused."""
    a = DE.Optimizer(20, 30, F=0.9, CR=0.9, xo="nec", obj="sphere", bounds=(-1.0, 1.0), seed=3,
                     params={"repair": "midpoint"})
    b = DE.Optimizer(20, 30, F=0.9, CR=0.9, xo="nec", obj="sphere", bounds=(-1.0, 1.0), seed=3)
    try:
        a.run(3)
        blob = a.save()
        with pytest.raises(DE.DEError) as e:
            b.load(blob)
        assert e.value.code == DE.DE_EINVAL
        a.load(blob)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("base", ["distinct", "random"])
def test_debug_mask_matches_oracle(xo, base):
    """de_debug_mask: the N x D mask of the next generation from the kernels'
    draw functions, row by row against the oracle's mask (Eq. 2, Alg. 8,
    Alg. 9 with Eq. 9) with the oracle's j_rand."""
    for (N, D, CR) in ((50, 37, 0.3), (20, 1001, 0.9), (8, 5, 1.0), (9, 64, 0.0)):
        opt, lo, hi = make(N, D, xo, "sphere", CR=CR, seed=41)
        try:
            opt.set_base(base)
            opt.run(2)
            g = opt.stats()["generation"]
            best = O.argmin(opt.population()[1])
            m = opt.debug_mask()
            for i in range(N):
                _, jr = O.donors_base(N, D, 41, g, i, base, best=best)
                ref, _ = O.mask(D, CR, xo, 41, g, i, jr)
                assert np.array_equal(m[i], ref), (xo, base, N, D, CR, i)
        finally:
            opt.close()


def test_debug_mask_batched_instance():
    specs = [dict(N=30 + 5 * k, D=D, F=0.5, CR=CR, xo=xo, obj="sphere", bounds=(-1.0, 1.0))
             for k, (D, CR, xo) in enumerate([(17, 0.9, "nec"), (300, 0.5, "bin"), (64, 0.8, "exp"),
                                             (2500, 0.9, "nec")])]
    bt = DE.Batch(specs, seed=43)
    try:
        bt.run(3)
        for k, s in enumerate(specs):
            g = bt.stats(k)["generation"]
            m = bt.debug_mask(k)
            for i in range(s["N"]):
                _, jr = O.donors(s["N"], s["D"], 43, g, i, inst=k)
                ref, _ = O.mask(s["D"], s["CR"], s["xo"], 43, g, i, jr, inst=k)
                assert np.array_equal(m[i], ref), (k, i)
    finally:
        bt.close()
