"""GPU parity of the shifted-rotated objectives (z = R (x - o)) against the
oracle, which evaluates them in FP64 from the same FP32 shift and rotation.

FP32 path: trials and draws bit-exact, FP32 fitness within 1e-5 relative of
FP64, selections identical outside the ambiguity band. The FP64 incumbent
re-evaluation agrees with the oracle's FP64 value to rounding."""
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


def make(N, D, xo, obj, prec="fp32", CR=0.9, F=0.5, seed=1, every=0, **extra):
    o = W.shift_vector(D, seed=2)
    R = W.rotation(D, seed=3)
    params = {"shift": o, "rotation": R, "prec": prec, "incumbent_every": every}
    params.update(extra)
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=W.BOXES[obj], seed=seed, params=params)
    return opt, o, R


def one_step(opt, o, R, xo, obj, F, CR, seed, repair="clip"):
    N, D = opt.N, opt.D
    lo, hi = W.BOXES[obj]
    pop = W.population(N, D, lo, hi, seed + 100)
    opt.set_population(pop)
    gp, gfit = opt.population()
    fit64 = O.evaluate(obj, pop, shift=o, rot=R)
    assert np.all(np.abs(gfit - fit64) <= tol(fit64)), "parent fitness"
    g = opt.stats()["generation"]
    trial, ft, acc, draws = opt.debug_step()
    s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, shift=o, rot=R, repair=repair)
    assert np.array_equal(draws, s.draws), "draws"
    assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32)), "trials"
    assert np.all(np.abs(ft - s.ftrial) <= tol(s.ftrial)), "trial fitness"
    amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
    assert np.array_equal(acc[~amb], s.accept[~amb]), "selection"
    np_, nf = opt.population()
    assert np.array_equal(np_.view(np.uint32), np.where(acc[:, None], trial, pop).view(np.uint32))
    return s, acc


@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("xo", ["nec", "bin", "exp"])
@pytest.mark.parametrize("N,D", [(64, 96), (40, 130), (300, 256), (20, 1024)])
def test_rotated_fp32_one_generation(obj, xo, N, D):
    opt, o, R = make(N, D, xo, obj, seed=7)
    try:
        one_step(opt, o, R, xo, obj, 0.5, 0.9, 7)
    finally:
        opt.close()


@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
def test_rotated_fp64_incumbent(obj):
    N, D = 50, 64
    opt, o, R = make(N, D, "nec", obj, seed=3, every=5)
    try:
        st = opt.stats()
        pop, fit = opt.population()
        assert st["incumbent_gen"] == 0
        ref = O.evaluate(obj, pop[st["best_index"]], shift=o, rot=R)
        assert st["incumbent_f64"] == pytest.approx(ref, rel=1e-12)
        opt.run(10)
        st = opt.stats()
        pop, fit = opt.population()
        assert st["incumbent_gen"] == 10 and st["generation"] == 10
        x, f, idx, bg = opt.best()
        ref = O.evaluate(obj, x, shift=o, rot=R)
        assert st["incumbent_f64"] == pytest.approx(ref, rel=1e-12)
        assert abs(f - ref) <= 1e-5 * max(1.0, abs(ref))
    finally:
        opt.close()


def test_rotated_identity_matches_plain_objective_shift():
    """R = I: the rotated Rastrigin of x equals the plain Rastrigin of x - o."""
    N, D = 32, 64
    o = W.shift_vector(D, seed=2)
    I = np.eye(D, dtype=np.float32)
    opt = DE.Optimizer(N, D, 0.5, 0.9, "nec", "sr_rastrigin", (-100.0, 100.0), seed=1,
                       params={"shift": o, "rotation": I})
    try:
        pop, fit = opt.population()
        ref = O.evaluate("rastrigin", (pop.astype(np.float64) - o.astype(np.float64)).astype(np.float32))
        assert np.all(np.abs(fit - ref) <= 1e-5 * np.maximum(1, np.abs(ref)))
    finally:
        opt.close()


# ---- the tensor-core paths: split BF16 / FP16 operands, interval decisions, FP32 re-evaluation --
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("N,D,xo,bound", [(256, 256, "nec", "probabilistic"), (300, 512, "bin", "probabilistic"),
                                          (128, 1024, "exp", "probabilistic"), (128, 512, "nec", "worst_case")])
def test_rotated_bf16_selections_equal_fp32_path(obj, N, D, xo, bound, prec):
    """Same seed and population on the FP32 path and a split-operand
    tensor-core path: identical trials and identical selections generation
    after generation."""
    a, o, R = make(N, D, xo, obj, prec="fp32", seed=5)
    b, _, _ = make(N, D, xo, obj, prec=prec, seed=5, bound=bound)
    try:
        lo, hi = W.BOXES[obj]
        pop = W.population(N, D, lo, hi, 55)
        a.set_population(pop)
        b.set_population(pop)
        reselected = 0
        for g in range(4):
            ta, fa, acca, da = a.debug_step()
            tb, fb, accb, db = b.debug_step()
            assert np.array_equal(da, db)
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.array_equal(acca, accb), "generation %d: selections differ" % g
            # BF16 values of decided rows are close to the FP32 path's; re-evaluated rows equal it
            rel = np.abs(fb.astype(np.float64) - fa) / np.maximum(1.0, np.abs(fa))
            assert rel.max() < 1e-3, rel.max()
            pa, ffa = a.population()
            pb, ffb = b.population()
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        st = b.stats()
        assert st["generation"] == 4 and st["reselected"] >= 0
        print("rows re-evaluated in FP32 over 4 generations:", st["reselected"], "of", 4 * N)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_rotated_bf16_against_oracle(prec):
    N, D, obj, xo = 200, 256, "sr_rastrigin", "nec"
    opt, o, R = make(N, D, xo, obj, prec=prec, seed=9)
    try:
        lo, hi = W.BOXES[obj]
        pop = W.population(N, D, lo, hi, 77)
        opt.set_population(pop)
        fit64 = O.evaluate(obj, pop, shift=o, rot=R)
        g = opt.stats()["generation"]
        trial, ft, acc, draws = opt.debug_step()
        s = O.step(pop, fit64, 0.5, 0.9, xo, obj, lo, hi, 9, g, shift=o, rot=R)
        assert np.array_equal(draws, s.draws)
        assert np.array_equal(trial.view(np.uint32), s.trial.view(np.uint32))
        assert np.all(np.abs(ft - s.ftrial) <= 1e-3 * np.maximum(1, np.abs(s.ftrial)))
        amb = np.abs(s.ftrial - fit64) <= tol(s.ftrial) + tol(fit64)
        assert np.array_equal(acc[~amb], s.accept[~amb])
    finally:
        opt.close()


# ---- the error bound that decides which split-operand selections are certain -----------------
U, UTC = 2.0 ** -24, 2.0 ** -23


def scale_exp(m):
    """s with m 2^s in [2^14, 2^15): the FP16 operands' power-of-two scaling."""
    s = 14 - int(np.floor(np.log2(m)))
    while m * 2.0 ** s >= 32768.0:
        s -= 1
    while m * 2.0 ** s < 16384.0:
        s += 1
    return s


def split_bound(prec, obj, D, o, R, box, trial, f, lam=8.0):
    """The probabilistic bound on |f_split - f_FP32| of each row, written out
    from its derivation: Hoeffding deviations of the operand-split residuals
    (unit roundoff u_s of the halves, plus FP16's subnormal floor), of the
    accumulation roundings (the leading product's D additions and the
    corrections' 2D on partial sums 2.01 u_s smaller), of the g evaluations
    and of the sums over k (each addition's error within u times its partial
    sum: 63 per 64-column tile and the tile sums on the FP32 path, 256 per
    256-column tile and the tile sums on the split path), the tensor cores'
    mean truncation (half an ulp per step: D/16 leading steps, 2D/16
    correction steps), and a second-order term. The 256-column tile sums come
    from an FP64 evaluation of the trial."""
    lo, hi = box
    o64 = o.astype(np.float64)
    amax = max(np.max(np.abs(lo - o64)), np.max(np.abs(hi - o64))) * (1 + 2.0 ** -22)
    if prec == "fp16":
        us = 2.0 ** -11
        fa = 2.0 ** (-25 - scale_exp(amax))
        fr = 2.0 ** (-25 - scale_exp(float(np.max(np.abs(R.astype(np.float64))))))
    else:
        us, fa, fr = 2.0 ** -8, 0.0, 0.0
    cs = 2.01 * us
    acc2 = UTC ** 2 * (1 + 2 * cs ** 2) + U ** 2
    a = (trial - o[None, :]).astype(np.float32).astype(np.float64)
    arow = np.abs(a).max(axis=1)                      # each row's own max |a_j|
    rep = (1.005 * us * us + fr * np.sqrt(D)) * arow + fa
    n2 = (a * a).sum(1)
    n = np.sqrt(n2)
    af = np.abs(f.astype(np.float64))
    if obj == "sr_elliptic":
        wmax = 10.0 ** 6
        H = 2 * np.sqrt(wmax * af)
        bias = (D / 16) * UTC * 2 * af
        g2half = wmax
    else:
        H = np.minimum(2 * n + 20 * np.pi * np.sqrt(D), (2 + 40 * np.pi ** 2) * n)   # |sin 2 pi z| <= 2 pi |z|
        bias = (D / 16) * UTC * n * H
        g2half = 1 + 20 * np.pi ** 2
    bias = 0.5 * (bias + (2 * D / 16) * UTC * cs * 4 * n * H)
    z = a @ R.astype(np.float64).T
    if obj == "sr_elliptic":
        g = 10.0 ** (6.0 * np.arange(D) / (D - 1)) * z * z
    else:
        g = z * z + 20.0 * np.sin(np.pi * z) ** 2
    tiles = g.reshape(g.shape[0], D // 256, 256).sum(axis=2)
    tsq = (tiles * tiles).sum(axis=1)
    s_rep = np.sqrt(3) * rep * H
    s_acc = 4 * np.sqrt(acc2) * n * H
    s_ev = U * (12 * af + np.sqrt(((63 + D // 64) * 1.21 + D // 256) * af * af + 256 * tsq))
    quad = g2half * 2 * D * (3 * rep ** 2 + acc2 * 16 * n2)
    return lam * np.sqrt(s_rep ** 2 + s_acc ** 2 + s_ev ** 2) + bias + quad


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("D", [256, 1024, 2048])
def test_rotated_bf16_error_within_bound(obj, D, prec):
    """Raw split-path values (almost no margin, so nearly every row is decided
    on them) against the FP32 path's values on the same parents and trials,
    at the start and after 100 generations: every row's difference stays well
    inside the bound the selection uses."""
    N = 1024
    a, o, R = make(N, D, "nec", obj, prec="fp32", seed=11)
    b, _, _ = make(N, D, "nec", obj, prec=prec, seed=11, margin_sigmas=1e-6)
    try:
        done = 0
        for G0 in (0, 100):
            a.run(G0 - done)
            b.run(G0 - done)
            done = G0
            pop, _ = a.population()
            a.set_population(pop)
            b.set_population(pop)
            ta, fa, _, _ = a.debug_step()
            tb, fb, _, _ = b.debug_step()
            done += 1
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            B = split_bound(prec, obj, D, o, R, W.BOXES[obj], tb, fb)
            r = np.abs(fb.astype(np.float64) - fa) / B
            print("%s D=%d %s gen %d: max |f_split - f_fp32| / bound = %.3f, mean signed (f_split - f_fp32) / bound "
                  "= %.3f" % (prec, D, obj, G0, r.max(), float(np.mean((fb.astype(np.float64) - fa) / B))))
            assert r.max() <= 0.25, r.max()
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("spread", [1e-2, 1e-5, 1e-7])
def test_rotated_split_near_the_optimum(obj, prec, spread):
    """A population within `spread` of the optimum o: |x - o| far below the
    box's reach, where FP16 remainders of 2^sa (x - o) fall into the
    subnormal range. The raw split values stay inside the bound (which counts
    that floor), and with the default margin the selections are the FP32
    path's, generation after generation."""
    N, D = 512, 256
    a, o, R = make(N, D, "nec", obj, prec="fp32", seed=21)
    b, _, _ = make(N, D, "nec", obj, prec=prec, seed=21)
    c, _, _ = make(N, D, "nec", obj, prec=prec, seed=21, margin_sigmas=1e-6)
    try:
        rng = np.random.default_rng(4)
        pop = (o[None, :].astype(np.float64) + spread * rng.uniform(-1.0, 1.0, size=(N, D))).astype(np.float32)
        for opt in (a, b, c):
            opt.set_population(pop)
        for g in range(3):
            ta, fa, acca, _ = a.debug_step()
            tb, fb, accb, _ = b.debug_step()
            tc, fc, _, _ = c.debug_step()
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.array_equal(ta.view(np.uint32), tc.view(np.uint32))
            assert np.array_equal(acca, accb), "generation %d: selections differ" % g
            B = split_bound(prec, obj, D, o, R, W.BOXES[obj], tc, fc)
            B = np.where(np.abs(tc - o[None, :]).max(axis=1) > 0, np.maximum(B, 1e-36), B)
            dif = np.abs(fc.astype(np.float64) - fa)
            assert np.all(dif[B == 0] == 0), "a = 0 exactly, yet the values differ"   # z = 0 on both paths
            r = np.where(B > 0, dif / np.where(B > 0, B, 1.0), 0.0)
            print("%s %s spread %g gen %d: max |f_split - f_fp32| / bound = %.3f" % (prec, obj, spread, g, r.max()))
            assert r.max() <= 0.25, r.max()
            c.set_population(a.population()[0])      # the raw-decision copy follows the FP32 path
        pa, _ = a.population()
        pb, _ = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        print("%s %s spread %g: rows re-evaluated in FP32: %d of %d" % (prec, obj, spread, b.stats()["reselected"],
                                                                       3 * N))
    finally:
        a.close()
        b.close()
        c.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
def test_rotated_bf16_lockstep_full_size(obj, prec):
    """The shifted-rotated workload at its full size (N = 4096, D = 1024):
    the split-operand path with its default bound makes the FP32 path's
    selections in every one of 30 generations, re-evaluating a small share of
    rows."""
    N, D, G = 4096, 1024, 30
    a, o, R = make(N, D, "nec", obj, prec="fp32", seed=1, every=10)
    b, _, _ = make(N, D, "nec", obj, prec=prec, seed=1, every=10)
    try:
        for g in range(G):
            ta, fa, acca, _ = a.debug_step()
            tb, fb, accb, _ = b.debug_step()
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32)), g
            assert np.array_equal(acca, accb), "generation %d: selections differ" % g
        sa, sb = a.stats(), b.stats()
        assert sa["accepts"] == sb["accepts"]
        assert sb["incumbent_gen"] == 30 and sa["incumbent_gen"] == 30
        pa, _ = a.population()
        pb, _ = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        x, f, idx, _ = b.best()
        ref = O.evaluate(obj, x, shift=o, rot=R)
        assert sb["incumbent_f64"] == pytest.approx(ref, rel=1e-12)
        print("%s %s: rows re-evaluated in FP32: %.2f%%" % (prec, obj, 100.0 * sb["reselected"] / (N * G)))
        assert sb["reselected"] < 0.2 * N * G
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("scale", [1e-3, 1e3])
def test_rotated_fp16_scaling_far_from_unit_boxes(obj, scale):
    """The FP16 operands' power-of-two scaling chosen for a box and shift
    scaled by 1e-3 and 1e3 (2^sa far from 1): the same trials and selections
    as the FP32 path over several generations."""
    N, D = 512, 256
    o = (W.shift_vector(D, seed=2).astype(np.float64) * scale).astype(np.float32)
    R = W.rotation(D, seed=3)
    box = (-100.0 * scale, 100.0 * scale)
    opts = []
    try:
        for prec in ("fp32", "fp16"):
            opts.append(DE.Optimizer(N, D, F=0.5, CR=0.9, xo="nec", obj=obj, bounds=box, seed=17,
                                     params={"shift": o, "rotation": R, "prec": prec}))
        pop = W.population(N, D, box[0], box[1], 19)
        for opt in opts:
            opt.set_population(pop)
        for g in range(4):
            ta, fa, acca, _ = opts[0].debug_step()
            tb, fb, accb, _ = opts[1].debug_step()
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.array_equal(acca, accb), "generation %d: selections differ" % g
            rel = np.abs(fb.astype(np.float64) - fa) / np.maximum(1e-30, np.abs(fa))
            assert np.median(rel) < 1e-5, np.median(rel)
        pa, _ = opts[0].population()
        pb, _ = opts[1].population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
    finally:
        for opt in opts:
            opt.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_rotated_long_ambiguous_list(prec):
    """A population within 1e-7 of the optimum at D = 1024 sends most rows,
    trial and parent, to the FP32 re-evaluation: over a thousand entries, more
    work items than the re-evaluation's resident groups, so each group walks
    several items. The re-evaluated values decide exactly as the FP32 path,
    and the populations stay bit-identical to its own."""
    N, D = 1024, 1024
    a, o, R = make(N, D, "nec", "sr_rastrigin", prec="fp32", seed=23)
    b, _, _ = make(N, D, "nec", "sr_rastrigin", prec=prec, seed=23)
    try:
        rng = np.random.default_rng(6)
        pop = (o[None, :].astype(np.float64) + 1e-7 * rng.uniform(-1.0, 1.0, size=(N, D))).astype(np.float32)
        a.set_population(pop)
        b.set_population(pop)
        most = 0
        for g in range(3):
            r0 = b.stats()["reselected"]
            ta, fa, acca, _ = a.debug_step()
            tb, fb, accb, _ = b.debug_step()
            assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
            assert np.array_equal(acca, accb), "generation %d: selections differ" % g
            most = max(most, b.stats()["reselected"] - r0)
        # 320 rows or more in one generation: 20 tiles of 16 entries x 16 column
        # tiles = 320 work items, more than the 2 x 152 resident groups
        print("%s: at most %d rows re-evaluated in one generation" % (prec, most))
        assert most >= 320, most
        pa, _ = a.population()
        pb, _ = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_rotated_checkpoint_resume(prec):
    """A split-path run saved after some generations and resumed in a fresh
    context continues bit for bit like the uninterrupted run (population,
    fitness, counters): the checkpoint carries the error bounds of the stored
    values, so split values are not taken as exact after the resume."""
    N, D = 512, 256
    a, o, R = make(N, D, "nec", "sr_rastrigin", prec=prec, seed=13)
    b, _, _ = make(N, D, "nec", "sr_rastrigin", prec=prec, seed=13)
    c, _, _ = make(N, D, "nec", "sr_rastrigin", prec="fp32", seed=13)
    try:
        a.run(7)
        blob = a.save()
        assert len(blob) == len(c.save()) + 4 * N          # the bounds: one float per row
        b.load(blob)
        b.prepare_run(9)                                    # graph only: the loaded state is kept
        a.run(9)
        b.run(9)
        pa, fa = a.population()
        pb, fb = b.population()
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
        sa, sb = a.stats(), b.stats()
        for k in ("generation", "accepts", "reselected", "best_gen"):
            assert sa[k] == sb[k], k
    finally:
        a.close()
        b.close()
        c.close()


def test_rotated_midpoint_repair():
    """The shifted-rotated path's trial kernel with DE_REPAIR_MIDPOINT (F = 1.4
    sends many mutants out of the box): trials bit for bit with the oracle,
    selections outside the ambiguity band (FP32 product)."""
    N, D, xo, obj = 64, 256, "nec", "sr_rastrigin"
    opt, o, R = make(N, D, xo, obj, prec="fp32", F=1.4, seed=5, repair="midpoint")
    try:
        one_step(opt, o, R, xo, obj, 1.4, 0.9, 5, repair="midpoint")
    finally:
        opt.close()
