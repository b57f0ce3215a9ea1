"""Eq. (9) and Alg. 8 on the GPU at the words where the answer changes.

Philox words land on a threshold of Eq. (9) with probability about
nT / 2^32 per row, so the generation tests never see one: an off-by-one in
the device lookup at a boundary between two consecutive L would pass them.
Here the device's NEC lookup (on the table in global memory, and on the copy
in shared memory that the pipelined kernel and the batched plans use) and
Alg. 8's continuation test are run through de_debug_lengths on chosen words:
every T_n - 1, T_n and T_n + 1 with T_n = ceil(Cr^n 2^32) (Cr^n the FP64
product, the reading of Eq. (9) the oracle follows), the words around
ceil(Cr 2^32), 0, 1, 2^32 - 1 and random words. Each is compared, bit for
bit, with the oracle (or_nec_length, or_exp_continues).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def boundary_words(Cr, D, n_random=2000, seed=0):
    """T_n - 1, T_n, T_n + 1 for every n < D with T_n > 1, plus the edges."""
    ws = {0, 1, 2, 2**31, 2**32 - 2, 2**32 - 1}
    if 0.0 < Cr < 1.0:
        c = Cr
        for _ in range(1, D):
            T = math.ceil(c * 2.0**32)          # c * 2^32 is exact: a power-of-two scaling
            if T <= 1:
                break
            ws.update((T - 1, T, T + 1))
            c = c * Cr                          # the FP64 product, rounded at each step
    Tc = math.ceil(Cr * 2.0**32)
    ws.update((Tc - 2, Tc - 1, Tc, Tc + 1))
    rng = np.random.default_rng(seed)
    ws.update(int(v) for v in rng.integers(0, 2**32, size=n_random, dtype=np.uint64))
    return np.array(sorted(w for w in ws if 0 <= w < 2**32), dtype=np.uint32)


def check_words(L_g, L_s, ec, words, Cr, D):
    want_L = np.array([O.nec_length(int(w), Cr, D) for w in words], dtype=np.int32)
    want_e = np.array([O.exp_continues(int(w), Cr) for w in words], dtype=bool)
    bad = np.nonzero(L_g != want_L)[0]
    assert bad.size == 0, ("global table", Cr, D, [(int(words[k]), int(L_g[k]), int(want_L[k])) for k in bad[:5]])
    bad = np.nonzero(L_s != want_L)[0]
    assert bad.size == 0, ("shared table", Cr, D, [(int(words[k]), int(L_s[k]), int(want_L[k])) for k in bad[:5]])
    assert np.array_equal(ec, want_e), ("exp", Cr, D)


@pytest.mark.parametrize("D", [10, 1000, 32768])
@pytest.mark.parametrize("Cr", [0.1, 0.5, 0.9, 0.99, 0.9999])
def test_nec_and_exp_lengths_at_threshold_words(Cr, D):
    _cuda()
    words = boundary_words(Cr, D)
    opt = DE.Optimizer(4, D, F=0.5, CR=Cr, xo="nec", obj="sphere", bounds=(-1.0, 1.0), seed=3)
    try:
        L_g, L_s, ec = opt.debug_lengths(words)
    finally:
        opt.close()
    check_words(L_g, L_s, ec, words, Cr, D)


@pytest.mark.parametrize("Cr", [0.0, 1.0, 2.0**-33, 1.0 - 2.0**-33])
def test_lengths_at_extreme_cr(Cr):
    """Cr = 0 (L = 1), Cr = 1 (L = D), and Cr one bit away from each end."""
    _cuda()
    D = 257
    words = boundary_words(Cr, D, n_random=500)
    opt = DE.Optimizer(4, D, F=0.5, CR=Cr, xo="nec", obj="sphere", bounds=(-1.0, 1.0), seed=3)
    try:
        L_g, L_s, ec = opt.debug_lengths(words)
    finally:
        opt.close()
    check_words(L_g, L_s, ec, words, Cr, D)


def test_batched_instance_lengths_at_threshold_words():
    """The per-instance tables and guess factors of a batch."""
    _cuda()
    specs = [dict(N=8, D=D, F=0.5, CR=Cr, xo="nec", obj="sphere", bounds=(-1.0, 1.0))
             for D, Cr in ((10, 0.1), (300, 0.5), (2000, 0.9), (1500, 0.99), (40, 0.999), (7, 0.0), (9, 1.0))]
    bt = DE.Batch(specs, seed=11)
    try:
        for k, s in enumerate(specs):
            words = boundary_words(s["CR"], s["D"], n_random=300, seed=k)
            L_g, L_s, ec = bt.debug_lengths(k, words)
            check_words(L_g, L_s, ec, words, s["CR"], s["D"])
    finally:
        bt.close()
