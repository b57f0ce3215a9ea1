"""Benchmark of the DE/rand/1 generation step on one GB300 (or N replicas).

Workload (default): the largest single-instance configuration, N = 16384
individuals x D = 10000 genes, FP32, F = 0.5, Cr = 0.9, Rosenbrock on
[-5.12, 5.12] with NEC (headline), plus binomial and classic exponential
crossover and the Ackley objective as side-by-side variants. Both population
buffers (0.66 GB each) exceed the 129 MB L2, so no flush is needed between
steps. One step = one generation = one launch of the fused generation kernel.

Prints ONE JSON line. Metric: individual-dims per second per generation
(N * D * steps / device time), with the HBM roofline fraction of the
generation kernel, a CPU-oracle baseline, an end-to-end figure through the C
ABI with host buffers, and the clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (different
seed); the value is the sum over ranks of N * D * K divided by the slowest
rank's time ("replicas only": one population has no natural row sharding).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "individual·dims/s per DE generation (NEC vs bin vs seq-exp), % of HBM roofline"
UNIT = "ind·dims/s"
WORKLOAD = "rosenbrock_ackley_N16384_D10000"
N_DEF, D_DEF, F_DEF, CR_DEF, SEED = 16384, 10000, 0.5, 0.9, 1
BOXES = {"rosenbrock": (-5.12, 5.12), "ackley": (-30.0, 30.0), "rastrigin": (-5.12, 5.12)}
FALLBACK_HBM_GBS = 6800.0
PROFILE = os.path.join(ROOT, "profiles", "gen_pipe_nec_rosenbrock_N16384_D10000.md")
KERNEL_SOURCES = ["common.cuh", "draws.cuh", "objectives.cuh", "gen_kernel.cuh", "gen_pipe.cuh", "ptx.cuh",
                  "philox.cuh"]


def kernel_fingerprint() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2101_06599_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (fingerprint match); else None."""
    try:
        with open(PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None
    fp, traffic = None, None
    for line in text.splitlines():
        line = line.strip().strip("`").strip()
        if line.startswith("kernel_fingerprint:"):
            fp = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch_full_size:"):
            try:
                traffic = float(line.split(":", 1)[1].strip())
            except ValueError:
                traffic = None
    return traffic if fp == kernel_fingerprint() else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(N, D, gens, d_accepts, d_masked):
    """Bytes a generation must move: every parent row (4 N D), the three donor
    genes of every masked gene (12 M), every accepted row (4 A D), and per row
    its fitness read, slot byte read and write (6 N) plus the fitness write of
    accepted rows (4 A)."""
    return 4.0 * N * D * gens + 12.0 * d_masked + 4.0 * d_accepts * D + 6.0 * N * gens + 4.0 * d_accepts


def time_variant(DE, torch, N, D, xo, obj, steps, warmup, seed, ramp_s=0.0, sampler=None):
    lo, hi = BOXES[obj]
    opt = DE.Optimizer(N, D, F=F_DEF, CR=CR_DEF, xo=xo, obj=obj, bounds=(lo, hi), seed=seed)
    try:
        s = opt.stream
        opt.run(warmup)
        if ramp_s > 0:
            t0 = time.time()
            while time.time() - t0 < ramp_s:
                opt.run(warmup)
                opt.synchronize()
        opt.prepare_run(steps)            # graph capture and instantiation: host set-up, not timed
        opt.synchronize()
        st0 = opt.stats()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        with timed_range(torch):
            ev0.record(s)
            opt.run(steps)
            ev1.record(s)
        ev1.synchronize()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        barrier()
        st1 = opt.stats()
        d_acc = st1["accepts"] - st0["accepts"]
        d_msk = st1["masked_genes"] - st0["masked_genes"]
        if opt.kernel() == 3:
            shape = "gen_stream_kernel<%s, %s>: one warp per row, 8 rows per CTA, chunks of 256 genes, " \
                    "winning trials recomputed and stored" % (xo.upper(), obj)
        elif opt.kernel() == 2:
            nc, stages, span, cps = opt.pipeline()
            shape = "gen_pipe_kernel<%s, %s>: %d CTA/SM, 1 producer warp + %d consumers, %d stages, " \
                    "donor spans of %d floats" % (xo.upper(), obj, cps, nc, stages, span)
        else:
            threads, vec = opt.launch()
            shape = "gen_kernel<%s, %s, vec4=%d> x %d threads/row" % (xo.upper(), obj, vec, threads)
        return opt, ms, d_acc, d_msk, shape
    except Exception:
        opt.close()
        raise


def time_batched(DE, torch, steps, warmup, seed, peak, n_inst=None, kernels="tuned"):
    """The 512-instance workload (D log-uniform in [10, 2000], N = min(10 D,
    4096), sphere/Rastrigin/Ackley/Rosenbrock round-robin, NEC, F = 0.5,
    Cr = 0.9), one generation of every instance per step. n_inst keeps the
    first n_inst instances (a smaller case of the same mix, for profiling).
    kernels: "tuned" (de_batch_autotune picks the row kernel per class of
    instances), or every instance on the streaming ("flow") or the staged
    ("staged") kernel."""
    from paper_2101_06599_gb300 import workloads as Wk
    specs = [dict(N=s.N, D=s.D, obj=s.objective, bounds=Wk.BOXES[s.objective], xo="nec", CR=CR_DEF, F=F_DEF)
             for s in Wk.batched_specs()]
    if n_inst:
        specs = specs[:n_inst]
    units = float(sum(s["N"] * s["D"] for s in specs))
    rows = float(sum(s["N"] for s in specs))
    b = DE.Batch(specs, seed=seed + 4)
    try:
        t_tune = time.time()
        if kernels == "tuned":
            groups = b.autotune(reps=3)
        else:
            b.set_groups([2 if kernels == "flow" else 1] * len(specs))
            groups = b.groups()
        t_tune = time.time() - t_tune
        def kind(g):
            return "staged" if g < 0 else ("streaming" if g == 2 else ("register" if g <= 32 else "cta"))
        kinds = sorted({kind(g) for g in groups})
        b.run(warmup)
        b.prepare_run(steps)
        b.synchronize()
        st0 = b.stats()
        acc0 = [b.stats(k)["accepts"] for k in range(len(specs))]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with timed_range(torch):
            ev0.record(b.stream)
            b.run(steps)
            ev1.record(b.stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        st1 = b.stats()
        acc_genes = sum((b.stats(k)["accepts"] - acc0[k]) * specs[k]["D"] for k in range(len(specs)))
    finally:
        b.close()
    d_acc = st1["accepts"] - st0["accepts"]
    d_msk = st1["masked_genes"] - st0["masked_genes"]
    # parent rows, donor genes of masked genes, accepted rows, per-row plans (written
    # and read, 32 bytes each), fitness and slot bytes
    byts = (4.0 * units * steps + 12.0 * d_msk + 4.0 * acc_genes + 64.0 * rows * steps
            + 6.0 * rows * steps + 4.0 * d_acc)
    gbs = byts / (ms / 1e3) / 1e9
    return {"workload": "batched_512_instances" if len(specs) == 512 else "batched_first_%d_instances" % len(specs),
            "instances": len(specs), "ind_dims_per_step": units,
            "value": units * steps / (ms / 1e3), "unit": UNIT, "ms_per_gen": ms / steps,
            "hbm_gbs": gbs, "frac": gbs / peak,
            # every instance on the staged, or every one on the streaming kernel: one
            # cooperative launch per generation
            "launches_per_step": 1 if kinds in (["staged"], ["streaming"]) else 2 + len(kinds),
            "row_kernels": {kd: sum(1 for g in groups if kind(g) == kd) for kd in kinds},
            "autotune_s": round(t_tune, 3),
            "a_acceptance": d_acc / (rows * steps), "m_masked_fraction": d_msk / (units * steps)}


def time_rotated(DE, torch, steps, warmup):
    """Shifted-rotated Rastrigin and elliptic (N = 4096, D = 1024, box
    [-100, 100], o ~ U[-80, 80] seed 2, Gaussian-QR rotation seed 3, NEC,
    F = 0.5, Cr = 0.9): the FP32-product path against the BF16 and FP16
    split-operand tensor-core paths with FP32 re-evaluation of uncertain
    selections; the runs start from the same population, so equal accept
    counts mean equal selections."""
    from paper_2101_06599_gb300 import workloads as Wk
    N, D = 4096, 1024
    o = Wk.shift_vector(D, seed=2)
    R = Wk.rotation(D, seed=3)
    out = {"workload": "shifted_rotated_N4096_D1024", "N": N, "D": D,
           "gemm_flop_per_gen": 2.0 * N * D * D}
    for obj in ("sr_rastrigin", "sr_elliptic"):
        r = {}
        for prec in ("fp32", "bf16", "fp16"):
            opt = DE.Optimizer(N, D, F=F_DEF, CR=CR_DEF, xo="nec", obj=obj, bounds=Wk.BOXES[obj], seed=SEED,
                               params={"shift": o, "rotation": R, "prec": prec, "incumbent_every": 50})
            try:
                opt.run(warmup)
                opt.prepare_run(steps)
                opt.synchronize()
                st0 = opt.stats()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                ev0.record(opt.stream)
                opt.run(steps)
                ev1.record(opt.stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
                st1 = opt.stats()
            finally:
                opt.close()
            r[prec] = {"ms_per_gen": ms / steps, "value": N * D * steps / (ms / 1e3),
                       "accepts": st1["accepts"] - st0["accepts"],
                       "reselected_frac": (st1["reselected"] - st0["reselected"]) / (N * steps)}
        r["speedup_bf16_over_fp32"] = r["fp32"]["ms_per_gen"] / r["bf16"]["ms_per_gen"]
        r["speedup_fp16_over_fp32"] = r["fp32"]["ms_per_gen"] / r["fp16"]["ms_per_gen"]
        r["same_selections"] = r["fp32"]["accepts"] == r["bf16"]["accepts"] == r["fp16"]["accepts"]
        out[obj] = r
    return out


def time_small_configs(DE, torch, warmup):
    """The small configurations: sphere N = 100, D = 30 for 200 generations
    (launch-bound, one graph of 200 generations) and Rastrigin N = 1024,
    D = 1000 (a 4 MB population that stays in L2) for 1000 generations at
    Cr in {0.1, 0.5, 0.9} with each crossover."""
    out = {}
    cases = [("sphere_N100_D30", 100, 30, "sphere", (-100.0, 100.0), [0.9], 200),
             ("rastrigin_N1024_D1000", 1024, 1000, "rastrigin", (-5.12, 5.12), [0.1, 0.5, 0.9], 1000)]
    for name, N, D, obj, box, crs, G in cases:
        res = {}
        for cr in crs:
            for xo in ("bin", "exp", "nec"):
                opt = DE.Optimizer(N, D, F=F_DEF, CR=cr, xo=xo, obj=obj, bounds=box, seed=SEED)
                try:
                    opt.run(G)                      # builds and warms the graph of G generations
                    opt.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(opt.stream)
                    opt.run(G)
                    ev1.record(opt.stream)
                    ev1.synchronize()
                    ms = ev0.elapsed_time(ev1)
                    best = opt.best()[1]
                finally:
                    opt.close()
                res["%s_cr%g" % (xo, cr)] = {"ms_per_gen": ms / G, "value": N * D * G / (ms / 1e3),
                                             "best_f": best}
        out[name] = {"generations": G, "results": res}
    return out


# Table I's CUDA columns (GTX 760, CuPy, seconds for Cr = 0.2 .. 1.0 x 100 runs): context only
PAPER_TABLE1_CUDA = {  # (D, Np): (CUDA-nec, CUDA-bin)
    (10, 100): (1.76, 6.99), (10, 1000): (1.18, 0.64), (10, 10000): (1.34, 0.94),
    (100, 100): (1.16, 0.66), (100, 1000): (1.23, 0.64), (100, 10000): (1.11, 1.36),
    (1000, 100): (0.66, 0.56), (1000, 1000): (1.07, 1.00), (1000, 10000): (4.31, 4.56),
    (10000, 100): (1.48, 0.97), (10000, 1000): (4.43, 3.91), (10000, 10000): (33.26, 39.14),
}


def time_crossover_grid(DE, torch, reps=100):
    """Crossover alone over Table I's grid: U = mask ? V : X on Np x D FP32
    matrices resident on the device (X, V seeded normal), 100 calls at each
    Cr in {0.2, 0.4, 0.6, 0.8, 1.0} (generation = call index), per crossover;
    the total seconds of the 500 calls (CUDA events, calls queued from
    Python) as Table I reports them, and the bytes moved per second on the
    device (12 bytes per gene: X and V read, U written)."""
    crs = (0.2, 0.4, 0.6, 0.8, 1.0)
    out = {"protocol": "de_crossover_apply, %d calls per Cr, Cr in %s" % (reps, list(crs)), "cells": []}
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for (D, Np), paper in PAPER_TABLE1_CUDA.items():
        x = torch.randn((Np, D), generator=g, device="cuda")
        v = torch.randn((Np, D), generator=g, device="cuda")
        u = torch.empty_like(x)
        cell = {"D": D, "Np": Np, "paper_gtx760_s": {"nec": paper[0], "bin": paper[1]}}
        s = torch.cuda.current_stream()
        for xo in ("nec", "bin", "exp"):
            for cr in crs[:1]:                          # warm-up (first launch of each kernel)
                DE.de_crossover_apply(u.data_ptr(), x.data_ptr(), v.data_ptr(), D, Np, D, cr, xo, SEED, 0,
                                      stream=s.cuda_stream)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(s)
            for cr in crs:
                for r in range(reps):
                    DE.de_crossover_apply(u.data_ptr(), x.data_ptr(), v.data_ptr(), D, Np, D, cr, xo, SEED, r,
                                          stream=s.cuda_stream)
            ev1.record(s)
            ev1.synchronize()
            sec = ev0.elapsed_time(ev1) / 1e3
            calls = reps * len(crs)
            cell[xo + "_s"] = sec
            cell[xo + "_gbs"] = 12.0 * Np * D * calls / sec / 1e9
        out["cells"].append(cell)
        del x, v, u
    return out


# The paper's DE workloads (its parameter table) and its CUDA-DE rows (GTX 760):
# (objective, D, Np, F, Cr, generations, box, Ackley constant), paper {crossover: (best value, best gen, s)}
PAPER_TABLE2 = [
    ("ackley", 1000, 500, 0.5, 0.2, 30000, (-30.0, 30.0), 0.02,
     {"nec": (2.62e-05, 29991, 323.97), "bin": (2.28e-04, 29983, 321.45)}),
    ("griewank", 500, 300, 0.25, 0.45, 20000, (-400.0, 400.0), 0.0,
     {"nec": (1.73e-16, 19936, 149.03), "bin": (2.22e-16, 6041, 143.95)}),
    ("rosenbrock", 50, 100, 0.65, 0.95, 10000, (-5.12, 5.12), 0.0,
     {"nec": (1.16e-07, 9996, 58.92), "bin": (9.93e-10, 10000, 56.72)}),
]


def time_paper_table2(DE, torch, chunk=1000):
    """The paper's three DE runs (Ackley 1000-D / 500 individuals / 30000
    generations with its printed inner constant 0.02, Griewank 500-D / 300 /
    20000 on [-400, 400], Rosenbrock 50-D / 100 / 10000) with NEC (DE/rand/1/L)
    and binomial crossover, under the distinct-donor rule and under the
    paper's random base rule (Alg. 3 with Alg. 6): total device time of all
    generations (graphs of `chunk` generations), best value and best
    generation. The best values are not a parity claim: the random streams
    differ from the paper's."""
    out = []
    for obj, D, Np, F, CR, G, box, b, paper in PAPER_TABLE2:
        for base in ("distinct", "random"):
          for xo in ("nec", "bin"):
            params = {"ackley_b": b} if b else None
            opt = DE.Optimizer(Np, D, F=F, CR=CR, xo=xo, obj=obj, bounds=box, seed=SEED, params=params)
            try:
                opt.set_base(base)
                opt.run(chunk)                            # warms the kernels; counted below from a fresh start
                opt.synchronize()
                opt.close()
                opt = DE.Optimizer(Np, D, F=F, CR=CR, xo=xo, obj=obj, bounds=box, seed=SEED, params=params)
                opt.set_base(base)
                opt.prepare_run(chunk)                    # graph set-up on the host, outside the timing
                opt.prepare_run(G % chunk)
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(opt.stream)
                done = 0
                while done < G:
                    k = min(chunk, G - done)
                    opt.run(k)
                    done += k
                ev1.record(opt.stream)
                ev1.synchronize()
                sec = ev0.elapsed_time(ev1) / 1e3
                st = opt.stats()
            finally:
                opt.close()
            out.append({"objective": obj, "D": D, "Np": Np, "F": F, "CR": CR, "generations": G,
                        "crossover": xo, "base": base, "seconds": sec, "us_per_gen": 1e6 * sec / G,
                        "value": Np * D * G / sec, "best_value": st["best_f"], "best_gen": st["best_gen"],
                        "paper_cuda_gtx760": {"best_value": paper[xo][0], "best_gen": paper[xo][1],
                                              "seconds": paper[xo][2]}})
    return out


_dist = None


def barrier():
    if _dist is not None:
        _dist.barrier()


class timed_range:
    """NVTX range "timed" around a timed region, so that a profiler can keep
    to the launches that are timed (ncu --nvtx --nvtx-include timed/)."""

    def __init__(self, torch):
        self.nvtx = getattr(torch.cuda, "nvtx", None)

    def __enter__(self):
        try:
            self.nvtx.range_push("timed")
        except Exception:
            self.nvtx = None
        return self

    def __exit__(self, *exc):
        if self.nvtx is not None:
            try:
                self.nvtx.range_pop()
            except Exception:
                pass
        return False


def _reduce(torch, v, op):
    if _dist is None:
        return v
    dev = "cuda" if _dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    _dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(torch, v):
    return _reduce(torch, v, _dist.ReduceOp.MAX) if _dist is not None else v


def sum_over_ranks(torch, v):
    return _reduce(torch, v, _dist.ReduceOp.SUM) if _dist is not None else v


def replica_seed(rank):
    """Rank r runs an independent replica from seed SEED + r."""
    return SEED + rank


def headline_config(N, D, obj, xo, world):
    """The workload description shared by the GPU line and the reference arm."""
    return {"workload": WORKLOAD if (N, D) == (N_DEF, D_DEF) and obj in ("rosenbrock", "ackley")
            else "%s_N%d_D%d" % (obj, N, D),
            "objective": obj, "crossover": xo, "N": N, "D": D,
            "F": F_DEF, "CR": CR_DEF, "parallelism": "replicas" if world > 1 else "single",
            "l2": ("inputs larger than L2 (two %.2f GB population buffers), no flush" % (4e-9 * N * D)
                   if 4.0 * N * D > 129e6 else
                   "population of %.1f MB fits in L2 (L2-resident case, no flush)" % (4e-6 * N * D))}


# ---- the CPU oracle on the host cores -----------------------------------------
# All-cores leg: P worker processes (spawned, so that none inherits a CUDA
# context) each run the single-threaded oracle on their own block of rows of
# the same generation; the population and fitness live in shared memory.
_W = {}


def _oracle_worker_init(shm_pop, shm_fit, N, D):
    from multiprocessing import shared_memory
    import oracle as O
    a = shared_memory.SharedMemory(name=shm_pop)
    b = shared_memory.SharedMemory(name=shm_fit)
    _W["shm"] = (a, b)
    _W["pop"] = np.ndarray((N, D), dtype=np.float32, buffer=a.buf)
    _W["fit"] = np.ndarray((N,), dtype=np.float64, buffer=b.buf)
    _W["O"] = O
    O.lib()


def _oracle_worker_rows(task):
    obj, xo, g, i0, i1 = task
    O = _W["O"]
    lo, hi = BOXES[obj]
    t0 = time.perf_counter()
    O.step(_W["pop"], _W["fit"], F_DEF, CR_DEF, xo, obj, lo, hi, SEED, g, rows=(i0, i1), want_trial=False)
    return time.perf_counter() - t0


def oracle_generation_rate_all_cores(pop, fit, obj, xo, rows_per_proc, steps, procs, budget_s=None):
    """Wall-clock rate of generations of the oracle over procs x rows_per_proc
    rows, one block of rows per process, every process a single-threaded
    oracle: `steps` generations, or (steps None) as many as fill budget_s.
    The generation index advances each step; the population is not advanced
    (each step starts from the same parents), which changes neither the work
    nor its cost. Returns (rate, seconds, steps)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    N, D = pop.shape
    a = shared_memory.SharedMemory(create=True, size=pop.nbytes)
    b = shared_memory.SharedMemory(create=True, size=fit.nbytes)
    try:
        np.ndarray(pop.shape, dtype=np.float32, buffer=a.buf)[:] = pop
        np.ndarray(fit.shape, dtype=np.float64, buffer=b.buf)[:] = fit
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(a.name, b.name, N, D)) as pool:
            pool.map(_oracle_worker_rows, [(obj, xo, 0, 0, 1)] * procs)           # start-up, not timed
            t0 = time.perf_counter()
            g = 0
            while (g < steps) if steps else (g == 0 or time.perf_counter() - t0 < budget_s):
                tasks = [(obj, xo, g, k * rows_per_proc, (k + 1) * rows_per_proc) for k in range(procs)]
                pool.map(_oracle_worker_rows, tasks, chunksize=1)
                g += 1
            secs = time.perf_counter() - t0
    finally:
        a.close(); a.unlink()
        b.close(); b.unlink()
    return procs * rows_per_proc * D * g / secs, secs, g


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_legs(N, D, obj, xo, budget_s, steps=None, warmup=0):
    """The oracle as it stands, single-threaded and on all host cores, on the
    same workload: returns the cpu_baseline object (all cores) with the
    single-thread figure beside it."""
    import oracle as O
    lo, hi = BOXES[obj]
    pop = O.init(N, D, lo, hi, SEED)
    fit = O.evaluate(obj, pop)
    rate1, rows1, timed1, secs1 = oracle_generation_rate(N, D, obj, xo, budget_s / 2, steps=steps, warmup=warmup,
                                                         pop=pop, fit=fit)
    procs = max(1, min(host_cores(), N))
    rows_p = max(1, min(rows1, N // procs))             # rows per process and step
    rate_p, secs_p, steps_p = oracle_generation_rate_all_cores(pop, fit, obj, xo, rows_p, steps, procs,
                                                               budget_s=budget_s / 2)
    return {"value": rate_p, "unit": UNIT, "cores": procs, "kind": "oracle", "ms_per_step": 1e3 * secs_p / steps_p,
            "sample": "%d generation(s) of the CPU oracle, %d processes x rows [k %d, (k+1) %d) of the same "
                      "N=%d x D=%d %s/%s workload (donors from all N rows), %.1f s wall, one single-threaded "
                      "oracle per process" % (steps_p, procs, rows_p, rows_p, N, D, obj, xo.upper(), secs_p),
            "single_thread": {"value": rate1, "cores": 1,
                              "sample": "%d generation(s) over rows [0, %d), %.1f s" % (timed1, rows1, secs1)}}


def oracle_generation_rate(N, D, obj, xo, budget_s, rows_per_step=None, steps=None, warmup=0, pop=None, fit=None):
    """Time the CPU oracle (single thread) on generations of the same workload.
    Returns (ind_dims_per_s, rows_per_step, steps_timed, seconds)."""
    import oracle as O
    lo, hi = BOXES[obj]
    if pop is None:
        pop = O.init(N, D, lo, hi, SEED)
        fit = O.evaluate(obj, pop)
    if rows_per_step is None:
        t0 = time.perf_counter()
        O.step(pop, fit, F_DEF, CR_DEF, xo, obj, lo, hi, SEED, 0, rows=(0, 64), want_trial=False)
        per_row = (time.perf_counter() - t0) / 64
        n_steps = steps if steps else 1
        rows_per_step = int(max(64, min(N, budget_s / max(n_steps, 1) / max(per_row, 1e-9))))
    g = 0
    for _ in range(warmup):
        r = O.step(pop, fit, F_DEF, CR_DEF, xo, obj, lo, hi, SEED, g, rows=(0, rows_per_step), want_trial=False)
        pop, fit, g = r.pop, r.fit, g + 1
    timed, t_tot = 0, 0.0
    target_steps = steps if steps else None
    while True:
        t0 = time.perf_counter()
        r = O.step(pop, fit, F_DEF, CR_DEF, xo, obj, lo, hi, SEED, g, rows=(0, rows_per_step), want_trial=False)
        t_tot += time.perf_counter() - t0
        pop, fit, g, timed = r.pop, r.fit, g + 1, timed + 1
        if target_steps is not None:
            if timed >= target_steps:
                break
        elif t_tot >= budget_s:
            break
    return rows_per_step * D * timed / t_tot, rows_per_step, timed, t_tot


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, warmup = args.steps, args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cpu = cpu_baseline_legs(N_DEF, D_DEF, "rosenbrock", "nec", 120.0, steps=steps, warmup=warmup)
    rate = cpu["value"]
    line = {
        "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
        "warmup": warmup, "ms_per_step": cpu["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 mutation, f64 fitness", "data": "synthetic",
        "impl": "reference",
        "config": headline_config(N_DEF, D_DEF, "rosenbrock", "nec", world),
        "cpu_baseline": cpu,
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-rotated", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=0,
                    help="batched leg: keep the first K of the 512 instances (profiling)")
    ap.add_argument("--batch-kernels", default="tuned", choices=["tuned", "flow", "staged"],
                    help="batched leg: row kernels picked by the autotuner, or one kernel for every instance")
    ap.add_argument("--no-crossover", action="store_true")
    ap.add_argument("--no-table2", action="store_true")
    ap.add_argument("--only", choices=["rotated", "small", "batched", "crossover", "table2"],
                    help="run one side workload alone (for profiling); prints its own JSON line")
    ap.add_argument("--N", type=int, default=N_DEF, help="rows (smaller cases for profiling)")
    ap.add_argument("--D", type=int, default=D_DEF, help="genes per row")
    ap.add_argument("--xo", default="nec", choices=["nec", "bin", "exp"],
                    help="headline crossover (other values are for profiling one kernel)")
    ap.add_argument("--obj", default="rosenbrock", choices=["rosenbrock", "ackley", "rastrigin"],
                    help="headline objective")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2101_06599_gb300 import de as DE

    global _dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        _dist = dist
    DE.load_library()
    N, D, K, W = args.N, args.D, args.steps, args.warmup
    seed = replica_seed(rank)

    if args.only:
        if args.only == "rotated":
            res = time_rotated(DE, torch, K, W)
        elif args.only == "small":
            res = time_small_configs(DE, torch, W)
        elif args.only == "crossover":
            res = time_crossover_grid(DE, torch)
        elif args.only == "table2":
            res = time_paper_table2(DE, torch)
        else:
            res = time_batched(DE, torch, K, W, seed, measured_hbm_peak()[0], args.batch_instances,
                               args.batch_kernels)
        if rank == 0:
            print(json.dumps({"only": args.only, "steps": K, "warmup": W, "result": res}))
        if _dist is not None:
            _dist.destroy_process_group()
        return 0

    # headline: NEC on Rosenbrock, clocks sampled across the ramp and the timed region
    with ClockSampler(local) as clk:
        opt, ms, d_acc, d_msk, shape = time_variant(DE, torch, N, D, args.xo, args.obj, K, W, seed,
                                                    ramp_s=1.0)
    ms_max = max_over_ranks(torch, ms)
    units = float(N) * D * K
    value = sum_over_ranks(torch, units) / (ms_max / 1e3)
    bytes_alg = algorithmic_bytes(N, D, K, d_acc, d_msk)
    avg_launch_s = ms / 1e3 / K
    peak, peak_src = measured_hbm_peak()
    achieved = bytes_alg / K / avg_launch_s / 1e9
    traffic = profiled_traffic() if (args.xo, args.obj, N, D) == ("nec", "rosenbrock", N_DEF, D_DEF) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_src,
                "kernel": shape,
                "algorithmic_bytes_per_launch": bytes_alg / K, "avg_launch_us": avg_launch_s * 1e6,
                "m_masked_fraction": d_msk / (N * D * K), "a_acceptance": d_acc / (N * K)}

    # end to end through the C ABI with host buffers: upload the population from
    # pinned memory (evaluated on the device), K generations, each step's best row
    # and value copied back into a pinned host record (de_best_async), then the
    # stream is drained and the last record read
    e2e = None
    if not args.no_e2e:
        from paper_2101_06599_gb300 import workloads as Wk
        host = torch.from_numpy(Wk.population(N, D, *BOXES[args.obj], seed + 1000)).pin_memory()
        host_np = host.numpy()
        rec = DE.best_record_bytes(D)
        ring = torch.empty(K * rec, dtype=torch.uint8).pin_memory().numpy()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        DE.de_set_population(opt.ctx, host_np, None)
        for k in range(K):
            DE.de_step(opt.ctx)
            DE.de_best_async(opt.ctx, ring[k * rec:(k + 1) * rec], D)
        DE.de_synchronize(opt.ctx)
        f_last, _, _, _ = DE.parse_best_record(ring[(K - 1) * rec:], D)
        t1 = time.perf_counter()
        firsts = [DE.parse_best_record(ring[k * rec:(k + 1) * rec], D)[0] for k in range(K)]
        assert all(b <= a for a, b in zip(firsts, firsts[1:])) and firsts[-1] == f_last
        e2e_s = max_over_ranks(torch, t1 - t0)
        e2e = {"value": sum_over_ranks(torch, units) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 4.0 * N * D / K, "d2h_bytes_per_step": float(rec),
               "job": "de_set_population(host pinned N x D) + %d x (de_step + de_best_async into a pinned "
                      "host record) + de_synchronize" % K}
    opt.close()

    variants = {}
    if not args.no_variants:
        for obj in ("rosenbrock", "ackley"):
            for xo in ("nec", "bin", "exp"):
                o2, ms2, a2, m2, sh2 = time_variant(DE, torch, N, D, xo, obj, K, W, seed)
                o2.close()
                b2 = algorithmic_bytes(N, D, K, a2, m2)
                ach2 = b2 / (ms2 / 1e3) / 1e9
                variants.setdefault(obj, {})[xo] = {
                    "value": units / (ms2 / 1e3), "ms_per_gen": ms2 / K, "hbm_gbs": ach2, "frac": ach2 / peak,
                    "m": m2 / (N * D * K), "a": a2 / (N * K), "kernel": sh2}

    batched = None
    if not args.no_batched:
        batched = time_batched(DE, torch, K, W, seed, peak, kernels=args.batch_kernels)

    rotated = None
    if not args.no_rotated:
        rotated = time_rotated(DE, torch, K, W)

    small = None
    if not args.no_small:
        small = time_small_configs(DE, torch, W)

    xgrid = None
    if not args.no_crossover:
        xgrid = time_crossover_grid(DE, torch)

    table2 = None
    if not args.no_table2:
        table2 = time_paper_table2(DE, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_legs(N, D, args.obj, args.xo, 24.0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": headline_config(N, D, args.obj, args.xo, world),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": K,
            "clocks": clk.summary(), "variants": variants, "batched": batched, "rotated": rotated,
            "small_configs": small, "crossover_table1": xgrid, "paper_table2": table2,
        }
        print(json.dumps(line))
    if _dist is not None:
        _dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
