"""GPU parity of the crossover-alone calls (de_crossover_mask,
de_crossover_apply) against the oracle's per-row mask: bit-exact masks and
trial matrices, padding untouched, and the draws equal to what de_step uses."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    DE.load_library()


def oracle_masks(N, D, Cr, xo, seed, g, inst=0, rows=None):
    rows = range(N) if rows is None else rows
    out = {}
    for i in rows:
        _, jrand = O.donors(max(N, 4), D, seed, g, i, inst)
        m, L = O.mask(D, Cr, xo, seed, g, i, jrand, inst)
        out[i] = m
    return out


CASES = [(37, 29, 0.9, 29), (64, 1000, 0.5, 1003), (20, 4097, 0.2, 4100), (16, 1, 0.9, 1), (50, 130, 0.0, 130),
         (33, 130, 1.0, 132), (8, 10000, 0.99, 10000), (40, 7, 0.6, 9)]


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("N,D,Cr,ld", CASES)
def test_crossover_mask_matches_oracle(xo, N, D, Cr, ld):
    import torch
    seed, g, inst = 31, 5, 3
    buf = torch.full((N, ld), 7, dtype=torch.uint8, device="cuda")
    DE.de_crossover_mask(buf.data_ptr(), ld, N, D, Cr, xo, seed, g, inst)
    torch.cuda.synchronize()
    got = buf.cpu().numpy()
    ref = oracle_masks(N, D, Cr, xo, seed, g, inst)
    for i in range(N):
        assert np.array_equal(got[i, :D], ref[i]), "row %d" % i
    assert np.all(got[:, D:] == 7), "padding written"


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
@pytest.mark.parametrize("N,D,Cr,ld", CASES)
def test_crossover_apply_matches_oracle(xo, N, D, Cr, ld):
    import torch
    seed, g = 77, 12
    rng = np.random.default_rng(1)
    x = rng.standard_normal((N, ld)).astype(np.float32)
    v = rng.standard_normal((N, ld)).astype(np.float32)
    tx, tv = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
    tu = torch.full((N, ld), -1.5, dtype=torch.float32, device="cuda")
    DE.de_crossover_apply(tu.data_ptr(), tx.data_ptr(), tv.data_ptr(), ld, N, D, Cr, xo, seed, g)
    torch.cuda.synchronize()
    u = tu.cpu().numpy()
    ref = oracle_masks(N, D, Cr, xo, seed, g)
    for i in range(N):
        exp = np.where(ref[i].astype(bool), v[i, :D], x[i, :D])
        assert np.array_equal(u[i, :D].view(np.uint32), exp.view(np.uint32)), "row %d" % i
    assert np.all(u[:, D:] == -1.5), "padding written"


def test_crossover_unaligned_buffers_take_the_scalar_path():
    """Bases off the 16-byte grid: same results through the element-wise path."""
    import torch
    N, D, ld, Cr, seed, g = 12, 203, 203, 0.7, 4, 2
    big = torch.zeros(N * ld + 3, dtype=torch.float32, device="cuda")
    x = torch.randn(N * ld + 1, dtype=torch.float32, device="cuda")
    v = torch.randn(N * ld + 1, dtype=torch.float32, device="cuda")
    DE.de_crossover_apply(big.data_ptr() + 4, x.data_ptr() + 4, v.data_ptr() + 4, ld, N, D, Cr, "bin", seed, g)
    mb = torch.zeros(N * ld + 1, dtype=torch.uint8, device="cuda")
    DE.de_crossover_mask(mb.data_ptr() + 1, ld, N, D, Cr, "bin", seed, g)
    torch.cuda.synchronize()
    u = big.cpu().numpy()[1:1 + N * ld].reshape(N, ld)
    xs = x.cpu().numpy()[1:].reshape(N, ld)
    vs = v.cpu().numpy()[1:].reshape(N, ld)
    m = mb.cpu().numpy()[1:].reshape(N, ld)
    ref = oracle_masks(N, D, Cr, "bin", seed, g)
    for i in range(N):
        assert np.array_equal(m[i], ref[i])
        assert np.array_equal(u[i], np.where(ref[i].astype(bool), vs[i], xs[i]))


@pytest.mark.parametrize("xo", ["bin", "exp", "nec"])
def test_crossover_mask_is_the_mask_de_step_uses(xo):
    """The trial of de_step differs from its parent only where the mask is set
    (and there it is the clipped mutant), for the same seed and generation."""
    import torch
    N, D, Cr, seed = 64, 300, 0.6, 9
    opt = DE.Optimizer(N, D, F=0.5, CR=Cr, xo=xo, obj="sphere", bounds=(-100.0, 100.0), seed=seed)
    try:
        opt.run(3)
        pop, _ = opt.population()
        g = opt.stats()["generation"]
        trial, _, _, draws = opt.debug_step()
        buf = torch.zeros((N, D), dtype=torch.uint8, device="cuda")
        DE.de_crossover_mask(buf.data_ptr(), D, N, D, Cr, xo, seed, g)
        torch.cuda.synchronize()
        m = buf.cpu().numpy().astype(bool)
        assert np.array_equal(trial[~m].view(np.uint32), pop[~m].view(np.uint32))
        assert np.array_equal(m.sum(1), draws[:, 4])    # binomial: the popcount; exp / NEC: L
    finally:
        opt.close()


def test_crossover_full_size_sampled_rows():
    """N = D = 10000 (the largest cell of the crossover timing grid): sampled rows."""
    import torch
    N, D, Cr, seed, g = 10000, 10000, 0.6, 5, 0
    buf = torch.empty((N, D), dtype=torch.uint8, device="cuda")
    for xo in ("bin", "nec"):
        DE.de_crossover_mask(buf.data_ptr(), D, N, D, Cr, xo, seed, g)
        torch.cuda.synchronize()
        rows = [0, 1, 4999, 9998, 9999]
        ref = oracle_masks(N, D, Cr, xo, seed, g, rows=rows)
        got = buf[rows].cpu().numpy()
        for k, i in enumerate(rows):
            assert np.array_equal(got[k], ref[i])
    del buf
