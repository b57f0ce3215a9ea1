"""The allocation-free NEC generation (de_nec_step_noalloc).

Some callers cannot call cudaMalloc: a plug-in inside a framework that owns
all device memory and only lends buffers, code that must not synchronise the
device (cudaMalloc and cudaFree may), a program with a fixed memory budget.
For them the library offers one generation on buffers the caller already
owns, with its scratch in a fixed array inside the library.

Checked here, through the C ABI:
- two such calls in a row (the second one consuming the first one's output)
  against de_step on a context holding the same population: bit-identical
  populations and fitness for D < 2048, where both run the same kernel; for
  D >= 2048 (de_step then sums the fitness in another order) identical trials,
  fitness within the suite's 1e-5 relative tolerance and the same selections
  outside that band;
- one call against the oracle's generation (Alg. 1): the same draws give the
  same trial rows bit for bit, and the same decisions wherever the two
  fitness values are not within tolerance of a tie;
- the device's free memory does not move across calls;
- sizes beyond the fixed scratch are refused.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def tol(f):
    return RTOL * np.maximum(1.0, np.abs(np.asarray(f, np.float64)))


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(torch, src_pop, src_fit, dst_pop, dst_fit, N, D, pitch, F, CR, obj, lo, hi, seed, g, stream):
    DE.de_nec_step_noalloc(src_pop.data_ptr(), src_fit.data_ptr(), dst_pop.data_ptr(), dst_fit.data_ptr(),
                           N, D, pitch, F, CR, obj, (lo, hi), seed, g, stream.cuda_stream)


@pytest.mark.parametrize("obj,N,D,CR", [("rastrigin", 256, 1000, 0.9), ("rosenbrock", 100, 33, 0.5),
                                        ("sphere", 64, 4096, 0.9)])
def test_noalloc_step_matches_context_twice(obj, N, D, CR):
    torch = _cuda()
    F, seed = 0.5, 5
    lo, hi = W.BOXES[obj]
    opt = DE.Optimizer(N, D, F=F, CR=CR, xo="nec", obj=obj, bounds=(lo, hi), seed=seed)
    try:
        pop0 = W.population(N, D, lo, hi, 77)
        opt.set_population(pop0)
        ref_pop, ref_fit = opt.population()
        g = opt.stats()["generation"]

        pitch = (D + 7) // 8 * 8
        dev = torch.device("cuda")
        bufs = [torch.zeros(N, pitch, dtype=torch.float32, device=dev) for _ in range(2)]
        fits = [torch.zeros(N, dtype=torch.float32, device=dev) for _ in range(2)]
        bufs[0][:, :D] = torch.from_numpy(ref_pop).to(dev)
        fits[0][:] = torch.from_numpy(ref_fit).to(dev)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()

        for call in range(2):
            src, dst = call % 2, (call + 1) % 2
            par_pop = bufs[src][:, :D].cpu().numpy()
            free_before = torch.cuda.mem_get_info()[0]
            _noalloc(torch, bufs[src], fits[src], bufs[dst], fits[dst], N, D, pitch, F, CR, obj, lo, hi, seed,
                     g + call, stream)
            torch.cuda.synchronize()
            if call > 0:          # the first call on a device may load the module's code
                assert torch.cuda.mem_get_info()[0] == free_before
            trial, ftrial, acc, _ = opt.debug_step()      # de_step's generation, with its trials
            ctx_pop, ctx_fit = opt.population()
            got_pop = bufs[dst][:, :D].cpu().numpy()
            got_fit = fits[dst].cpu().numpy()
            if D < 2048:
                assert np.array_equal(got_pop.view(np.uint32), ctx_pop.view(np.uint32)), "population differs"
                assert np.array_equal(got_fit.view(np.uint32), ctx_fit.view(np.uint32)), "fitness differs"
            else:
                same = np.all(got_pop.view(np.uint32) == ctx_pop.view(np.uint32), axis=1)
                took = ~np.all(got_pop.view(np.uint32) == par_pop.view(np.uint32), axis=1)
                # every row holds either the parent or de_step's trial, bit for bit
                assert np.all(same | np.all(got_pop.view(np.uint32) == trial.view(np.uint32), axis=1)
                              | ~took)
                assert np.all(np.abs(got_fit.astype(np.float64) - ctx_fit) <= tol(ctx_fit)), "fitness differs"
                # a differing selection needs the trial and the parent within tolerance of a tie
                diff = ~same
                assert np.all(np.abs(ftrial[diff].astype(np.float64) - ref_fit[diff]) <= 2 * tol(ref_fit[diff]))
            # continue both from the context's population so that the next call compares like with like
            bufs[dst][:, :D] = torch.from_numpy(ctx_pop).to(dev)
            fits[dst][:] = torch.from_numpy(ctx_fit).to(dev)
            ref_fit = ctx_fit
            torch.cuda.synchronize()
    finally:
        opt.close()


@pytest.mark.parametrize("obj,N,D,CR", [("ackley", 40, 130, 0.9), ("griewank", 33, 29, 0.1),
                                        ("elliptic", 6, 4099, 0.9999)])
def test_noalloc_step_matches_oracle(obj, N, D, CR):
    torch = _cuda()
    F, seed, g = 0.5, 9, 3
    lo, hi = W.BOXES[obj]
    pop = W.population(N, D, lo, hi, 5)
    fit64 = O.evaluate(obj, pop)
    fit32 = fit64.astype(np.float32)
    pitch = (D + 7) // 8 * 8
    dev = torch.device("cuda")
    src = torch.zeros(N, pitch, dtype=torch.float32, device=dev)
    dst = torch.zeros(N, pitch, dtype=torch.float32, device=dev)
    src[:, :D] = torch.from_numpy(pop).to(dev)
    fsrc = torch.from_numpy(fit32).to(dev)
    fdst = torch.zeros(N, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for call in range(2):            # the same generation twice: the scratch left by the first call is reset
        _noalloc(torch, src, fsrc, dst, fdst, N, D, pitch, F, CR, obj, lo, hi, seed, g, stream)
        torch.cuda.synchronize()
        got_pop = dst[:, :D].cpu().numpy()
        got_fit = fdst.cpu().numpy()
        ref = O.step(pop, fit64, F, CR, "nec", obj, lo, hi, seed, g)
        took = ~np.all(got_pop.view(np.uint32) == pop.view(np.uint32), axis=1)
        # an accepted row is the oracle's trial bit for bit, with its fitness within tolerance
        assert np.array_equal(got_pop[took].view(np.uint32), ref.trial[took].view(np.uint32))
        assert np.all(np.abs(got_fit[took].astype(np.float64) - ref.ftrial[took]) <= tol(ref.ftrial[took]))
        assert np.array_equal(got_fit[~took].view(np.uint32), fit32[~took].view(np.uint32))
        # decisions: identical unless the trial and the parent are within tolerance of a tie
        clear = np.abs(ref.ftrial - fit64) > tol(ref.ftrial) + tol(fit64)
        assert np.array_equal(took[clear], ref.accept[clear])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = _cuda()
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    b = torch.zeros(16, dtype=torch.float32, device="cuda")
    c = torch.zeros(16, dtype=torch.float32, device="cuda")
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    for N, D in ((65537, 4), (8, 32769), (3, 4)):
        with pytest.raises(DE.DEError) as e:
            DE.de_nec_step_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), d.data_ptr(), N, D,
                                   (D + 3) // 4 * 4, 0.5, 0.9, "sphere", (-1.0, 1.0), 1, 0)
        assert e.value.code == DE.DE_EINVAL
