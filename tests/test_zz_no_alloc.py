"""The allocation-free NEC generation (de_nec_step_noalloc) against the
context API.

Some callers cannot call cudaMalloc — a plug-in inside a framework that owns
all device memory, code that must not synchronise the device, a program with
a fixed memory budget — so the library offers one generation on buffers the
caller already owns, with its scratch in a fixed array inside the library.
This test runs two such calls in a row (the second one consuming the first
one's output) and checks each against de_step on a context holding the same
population: populations equal, FP32 fitness within the suite's 1e-5 relative
tolerance (rows may only differ where the two decisions were within that
tolerance of a tie). It also checks that the calls leave the device's free
memory unchanged. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def tol(f):
    return RTOL * np.maximum(1.0, np.abs(np.asarray(f, np.float64)))


@pytest.mark.parametrize("obj,N,D,CR", [("rastrigin", 256, 1000, 0.9), ("rosenbrock", 100, 33, 0.5)])
def test_noalloc_step_matches_context_twice(obj, N, D, CR):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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
            free_before = torch.cuda.mem_get_info()[0]
            DE.de_nec_step_noalloc(bufs[src].data_ptr(), fits[src].data_ptr(), bufs[dst].data_ptr(),
                                   fits[dst].data_ptr(), N, D, pitch, F, CR, obj, (lo, hi), seed, g + call,
                                   stream.cuda_stream)
            torch.cuda.synchronize()
            if call > 0:          # the first call on a device may load the module's code
                assert torch.cuda.mem_get_info()[0] == free_before
            opt.step()
            ctx_pop, ctx_fit = opt.population()
            got_pop = bufs[dst][:, :D].cpu().numpy()
            got_fit = fits[dst].cpu().numpy()
            assert np.all(np.abs(got_fit.astype(np.float64) - ctx_fit) <= tol(ctx_fit)), "fitness differs"
            same = np.all(got_pop.view(np.uint32) == ctx_pop.view(np.uint32), axis=1)
            assert np.all(np.abs(got_fit[~same].astype(np.float64) - ctx_fit[~same]) <= tol(ctx_fit[~same]))
            assert same.mean() > 0.99
            # continue both from the context's population so that the next call compares like with like
            bufs[dst][:, :D] = torch.from_numpy(ctx_pop).to(dev)
            fits[dst][:] = torch.from_numpy(ctx_fit).to(dev)
            torch.cuda.synchronize()
    finally:
        opt.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    b = torch.zeros(16, dtype=torch.float32, device="cuda")
    c = torch.zeros(16, dtype=torch.float32, device="cuda")
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    for N, D in ((65537, 4), (8, 32769), (3, 4)):
        with pytest.raises(DE.DEError) as e:
            DE.de_nec_step_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), d.data_ptr(), N, D,
                                   (D + 3) // 4 * 4, 0.5, 0.9, "sphere", (-1.0, 1.0), 1, 0)
        assert e.value.code == DE.DE_EINVAL
