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


def make(N, D, xo, obj, prec="fp32", CR=0.9, F=0.5, seed=1, every=0):
    o = W.shift_vector(D, seed=2)
    R = W.rotation(D, seed=3)
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo=xo, obj=obj, bounds=W.BOXES[obj], seed=seed,
                       params={"shift": o, "rotation": R, "prec": prec, "incumbent_every": every})
    return opt, o, R


def one_step(opt, o, R, xo, obj, F, CR, seed):
    N, D = opt.N, opt.D
    lo, hi = W.BOXES[obj]
    pop = W.population(N, D, lo, hi, seed + 100)
    opt.set_population(pop)
    gp, gfit = opt.population()
    fit64 = O.evaluate(obj, pop, shift=o, rot=R)
    assert np.all(np.abs(gfit - fit64) <= tol(fit64)), "parent fitness"
    g = opt.stats()["generation"]
    trial, ft, acc, draws = opt.debug_step()
    s = O.step(pop, fit64, F, CR, xo, obj, lo, hi, seed, g, shift=o, rot=R)
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


# ---- the tensor-core path: split BF16 operands, interval decisions, FP32 re-evaluation ---------
@pytest.mark.parametrize("obj", ["sr_rastrigin", "sr_elliptic"])
@pytest.mark.parametrize("N,D,xo", [(256, 256, "nec"), (300, 512, "bin"), (128, 1024, "exp")])
def test_rotated_bf16_selections_equal_fp32_path(obj, N, D, xo):
    """Same seed and population on the FP32 path and the BF16 tensor-core path:
    identical trials and identical selections generation after generation."""
    a, o, R = make(N, D, xo, obj, prec="fp32", seed=5)
    b, _, _ = make(N, D, xo, obj, prec="bf16", seed=5)
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


def test_rotated_bf16_against_oracle():
    N, D, obj, xo = 200, 256, "sr_rastrigin", "nec"
    opt, o, R = make(N, D, xo, obj, prec="bf16", seed=9)
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
