"""Failure paths, made to happen without faulting the GPU.

- A device wait that runs out: the grid barrier of the batched one-launch
  generation (it guards no copy or MMA in flight) is given a 1 ns limit with
  de_set_wait_limit, so the CTAs that reach it first give up. The next
  synchronising call must report DE_ETIMEOUT, later launches must be refused
  with DE_ESTATE, and the generations that ran must still be complete: the
  populations equal those of the same batch run with the default limit, bit
  for bit, and the oracle's generation.
- An allocation that fails: the allocator hook returns NULL on its k-th call,
  for every k a successful create makes. Each create must return DE_ENOMEM
  and hand every block it got back to the allocator; a debug step whose
  scratch allocation fails returns DE_ENOMEM and leaves the context usable.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_06599_gb300 import de as DE
from paper_2101_06599_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _specs():
    rng = np.random.default_rng(21)
    specs = []
    for k in range(48):
        D = int(round(np.exp(rng.uniform(np.log(10), np.log(600)))))
        obj = ["sphere", "rastrigin", "ackley", "rosenbrock"][k % 4]
        specs.append(dict(N=min(10 * D, 1024), D=D, F=0.5, CR=0.9, xo="nec", obj=obj, bounds=W.BOXES[obj]))
    return specs


def test_barrier_timeout_is_reported_refuses_launches_and_keeps_the_generation_whole():
    _cuda()
    specs = _specs()
    a = DE.Batch(specs, seed=13)
    b = DE.Batch(specs, seed=13)
    try:
        assert a.wait_limit() == 1_000_000_000
        starts = [a.population(k) for k in range(len(specs))]
        a.set_wait_limit(1)
        assert a.wait_limit() == 1
        G = 4
        for _ in range(G):
            a.step()
            b.step()
        with pytest.raises(DE.DEError) as e:
            a.synchronize()
        assert e.value.code == DE.DE_ETIMEOUT
        with pytest.raises(DE.DEError) as e:
            a.step()
        assert e.value.code == DE.DE_ESTATE
        with pytest.raises(DE.DEError) as e:
            a.run(3)
        assert e.value.code == DE.DE_ESTATE
        b.synchronize()
        for k in range(len(specs)):
            pa, fa = a.population(k)
            pb, fb = b.population(k)
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32)), k
            assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32)), k
        # the first generation of a few instances against the oracle, from the shared start
        c = DE.Batch(specs, seed=13)
        try:
            c.set_wait_limit(1)
            c.step()
            for k in (0, 5, 17, 46):
                s = specs[k]
                lo, hi = s["bounds"]
                pop0, fit0 = starts[k]
                ref = O.step(pop0, O.evaluate(s["obj"], pop0), s["F"], s["CR"], "nec", s["obj"], lo, hi, 13, 0,
                             inst=k)
                got, _ = c.population(k)
                f0 = O.evaluate(s["obj"], pop0)
                same = np.all(got.view(np.uint32) == ref.pop.view(np.uint32), axis=1)
                # rows may differ only where the FP32 and FP64 decisions are within tolerance of a tie
                t = 1e-5 * (np.maximum(1.0, np.abs(ref.ftrial)) + np.maximum(1.0, np.abs(f0)))
                assert np.all(np.abs(ref.ftrial[~same] - f0[~same]) <= t[~same]), k
                assert same.mean() > 0.9, k
        finally:
            c.close()
    finally:
        a.close()
        b.close()


def test_wait_limit_arguments():
    _cuda()
    bt = DE.Batch(_specs()[:3], seed=1)
    try:
        with pytest.raises(DE.DEError) as e:
            bt.set_wait_limit(-1)
        assert e.value.code == DE.DE_EINVAL
        bt.set_wait_limit(5000)
        assert bt.wait_limit() == 5000
        bt.set_wait_limit(0)
        assert bt.wait_limit() == 1_000_000_000
        bt.step()
        bt.synchronize()               # the default limit never runs out here
    finally:
        bt.close()


class _FailingAllocator:
    """Device blocks from torch; the k-th request (1-based) gets NULL."""

    def __init__(self, torch):
        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail_at = None
        self.a = DE._ALLOC_FN(self._alloc)
        self.f = DE._FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, nbytes, stream, user):
        assert ptr in self.live, "freed a block it was not given"
        del self.live[ptr]

    def install(self):
        assert DE.load_library().de_set_allocator(self.a, self.f, None) == DE.DE_OK

    def arm(self, k):
        self.calls = 0
        self.fail_at = k


def _creators(torch):
    s = torch.cuda.Stream()
    rng = np.random.default_rng(3)
    D = 128
    shift = rng.uniform(-80, 80, D).astype(np.float32)
    q, r = np.linalg.qr(rng.standard_normal((D, D)))
    rot = (q * np.sign(np.diag(r))).astype(np.float32)
    return {
        "nec": lambda: DE.de_create(64, 300, 0.5, 0.9, "nec", "rastrigin", (-5.12, 5.12), 1, None, s.cuda_stream),
        "bin_wide": lambda: DE.de_create(16, 4096, 0.5, 0.9, "bin", "sphere", (-100.0, 100.0), 1, None,
                                         s.cuda_stream),
        "rotated": lambda: DE.de_create(128, D, 0.5, 0.9, "nec", "sr_rastrigin", (-100.0, 100.0), 1,
                                        dict(shift=shift, rotation=rot, prec="fp32"), s.cuda_stream),
        "batch": lambda: DE.de_batch_create([dict(N=40, D=30, obj="sphere", bounds=(-1.0, 1.0)),
                                             dict(N=20, D=3000, xo="bin", obj="ackley", bounds=(-30.0, 30.0))],
                                            1, s.cuda_stream),
    }


@pytest.mark.parametrize("kind", ["nec", "bin_wide", "rotated", "batch"])
def test_allocation_failure_returns_enomem_and_frees_everything(kind):
    torch = _cuda()
    fa = _FailingAllocator(torch)
    make = _creators(torch)[kind]
    fa.install()
    try:
        fa.arm(None)
        h = make()
        n = fa.calls
        assert n >= 3 and fa.live
        DE.de_destroy(h)
        assert not fa.live
        for k in range(1, n + 1):
            fa.arm(k)
            with pytest.raises(DE.DEError) as e:
                make()
            assert e.value.code == DE.DE_ENOMEM, (kind, k)
            assert not fa.live, (kind, k, len(fa.live))
        # the debug step's scratch: its allocation fails, the context carries on
        if kind in ("nec", "bin_wide"):
            fa.arm(None)
            h = make()
            try:
                N, D = (64, 300) if kind == "nec" else (16, 4096)
                fa.arm(1)
                out = np.empty((N, D), np.float32)
                with pytest.raises(DE.DEError) as e:
                    DE.de_debug_step(h, out, None, None, None)
                assert e.value.code == DE.DE_ENOMEM
                fa.arm(None)
                DE.de_step(h)
                DE.de_synchronize(h)
            finally:
                DE.de_destroy(h)
            assert not fa.live
    finally:
        DE.use_torch_allocator(True)
