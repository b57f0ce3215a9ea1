"""Plain CPU oracle for one DE/rand/1 generation (arXiv 2101.06599).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product (``paper_2101_06599_gb300``) never imports it, and the C
source here shares no code, header or table with the CUDA library.

The arithmetic lives in ``de_oracle.c`` (plain C11, FP32 mutation with
contraction off, FP64 fitness). This module builds it with gcc and wraps it
with ctypes, taking and returning numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "de_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

XO = {"bin": 0, "exp": 1, "nec": 2}
OBJ = {"sphere": 0, "rastrigin": 1, "ackley": 2, "rosenbrock": 3,
       "griewank": 4, "elliptic": 5, "sr_rastrigin": 6, "sr_elliptic": 7}
STREAM = {"init": 0, "idx": 1, "len": 2, "bin": 3, "exp": 4}


def build(force: bool = False) -> str:
    """Compile de_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FP contraction)."""
    srcs = [_SRC, os.path.join(_HERE, "de_oracle.h")]
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in srcs)):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u32p = C.POINTER(C.c_uint32)
        i32p = C.POINTER(C.c_int32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_word.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int32, C.c_uint32]
        L.or_word.restype = C.c_uint32
        L.or_donors.argtypes = [C.c_int32, C.c_int32, C.c_uint64, C.c_uint32, C.c_int64,
                                C.c_int32, i32p, i32p]
        L.or_donors.restype = None
        L.or_nec_length.argtypes = [C.c_uint32, C.c_double, C.c_int32]
        L.or_nec_length.restype = C.c_int32
        L.or_exp_continues.argtypes = [C.c_uint32, C.c_double]
        L.or_exp_continues.restype = C.c_int
        L.or_exp_length.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int32, C.c_double, C.c_int32]
        L.or_exp_length.restype = C.c_int32
        L.or_mask.argtypes = [C.c_int32, C.c_double, C.c_int, C.c_uint64, C.c_uint32, C.c_int64,
                              C.c_int32, C.c_int32, C.c_void_p]
        L.or_mask.restype = C.c_int32
        L.or_eval.argtypes = [C.c_int, C.c_int32, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        L.or_eval.restype = C.c_double
        L.or_init.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_uint64, C.c_uint32,
                              C.c_void_p]
        L.or_init.restype = None
        L.or_step.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_double, C.c_int, C.c_int,
                              C.c_float, C.c_float, C.c_uint64, C.c_uint32, C.c_int64,
                              C.c_double, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_int32, C.c_int32,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_step.restype = C.c_int
        L.or_argmin.argtypes = [C.c_int32, C.c_void_p]
        L.or_argmin.restype = C.c_int32
        L.or_step_base.argtypes = L.or_step.argtypes + [C.c_int, C.c_int32, C.c_int]
        L.or_step_base.restype = C.c_int
        L.or_donors_base.argtypes = [C.c_int32, C.c_int32, C.c_uint64, C.c_uint32, C.c_int64, C.c_int32,
                                     C.c_int, C.c_int32, C.c_void_p, C.c_void_p]
        L.or_donors_base.restype = None
        L.or_base_offset.argtypes = [C.c_int32, C.c_uint64, C.c_uint32, C.c_int64]
        L.or_base_offset.restype = C.c_int32
        L.or_base_perm.argtypes = [C.c_int32, C.c_uint64, C.c_uint32, C.c_int64, C.c_int32]
        L.or_base_perm.restype = C.c_int32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def philox(ctr, key):
    """Philox4x32-10 block function: 4 counter words, 2 key words -> 4 words."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def word(seed, inst, stream, g, i, idx):
    s = STREAM[stream] if isinstance(stream, str) else int(stream)
    return int(lib().or_word(seed, inst, s, g, i, idx))


def donors(N, D, seed, g, i, inst=0):
    r = (C.c_int32 * 3)()
    j = C.c_int32()
    lib().or_donors(N, D, seed, inst, g, i, r, C.byref(j))
    return (int(r[0]), int(r[1]), int(r[2])), int(j.value)


BASE = {"distinct": 0, "random": 1, "offset": 2, "permutation": 3, "best": 4}
REPAIR = {"clip": 0, "midpoint": 1}


def donors_base(N, D, seed, g, i, base, best=0, inst=0):
    """(r0, r1, r2) and j_rand of row i under a base index rule."""
    r = (C.c_int32 * 3)()
    j = C.c_int32()
    lib().or_donors_base(N, D, seed, inst, g, i, BASE[base] if isinstance(base, str) else int(base), best,
                         r, C.byref(j))
    return (int(r[0]), int(r[1]), int(r[2])), int(j.value)


def base_offset(N, seed, g, inst=0):
    return int(lib().or_base_offset(N, seed, inst, g))


def base_perm(N, seed, g, i, inst=0):
    return int(lib().or_base_perm(N, seed, inst, g, i))


def nec_length(w, Cr, D):
    return int(lib().or_nec_length(int(w) & 0xFFFFFFFF, float(Cr), int(D)))


def exp_continues(w, Cr):
    """Alg. 8's continuation test for one word: w / 2^32 < Cr."""
    return bool(lib().or_exp_continues(int(w) & 0xFFFFFFFF, float(Cr)))


def exp_length(seed, g, i, Cr, D, inst=0):
    return int(lib().or_exp_length(seed, inst, g, i, float(Cr), D))


def mask(D, Cr, xo, seed, g, i, jrand, inst=0):
    m = np.zeros(D, dtype=np.uint8)
    L = lib().or_mask(D, float(Cr), XO[xo], seed, inst, g, i, jrand, _ptr(m))
    return m, int(L)


def evaluate(obj, x, ackley_b=0.2, shift=None, rot=None):
    """FP64 objective value(s); x is a D-vector or an N x D array."""
    x = _f32(x)
    o = OBJ[obj] if isinstance(obj, str) else int(obj)
    shift, rot = _f32(shift), _f32(rot)
    if x.ndim == 1:
        return float(lib().or_eval(o, x.shape[0], _ptr(x), ackley_b, _ptr(shift), _ptr(rot)))
    D = x.shape[1]
    out = np.empty(x.shape[0], dtype=np.float64)
    for i in range(x.shape[0]):
        row = np.ascontiguousarray(x[i])
        out[i] = lib().or_eval(o, D, _ptr(row), ackley_b, _ptr(shift), _ptr(rot))
    return out


def init(N, D, lo, hi, seed, inst=0):
    pop = np.empty((N, D), dtype=np.float32)
    lib().or_init(N, D, lo, hi, seed, inst, _ptr(pop))
    return pop


def argmin(fit):
    fit = np.ascontiguousarray(fit, dtype=np.float64)
    return int(lib().or_argmin(fit.shape[0], _ptr(fit)))


class StepResult:
    """Outputs of one oracle generation over rows [i0, i1)."""

    def __init__(self, pop, fit, draws, trial, ftrial, accept, mask):
        self.pop, self.fit = pop, fit
        self.draws, self.trial, self.ftrial = draws, trial, ftrial
        self.accept, self.mask = accept, mask

    @property
    def r(self):
        return self.draws[:, 0:3]

    @property
    def jrand(self):
        return self.draws[:, 3]

    @property
    def L(self):
        return self.draws[:, 4]


def step(pop, fit, F, Cr, xo, obj, lo, hi, seed, g, inst=0, ackley_b=0.2,
         shift=None, rot=None, rows=None, want_trial=True, want_mask=False, base="distinct", best=None,
         repair="clip"):
    """One generation of Alg. 1 (rows `rows` = (i0, i1), default all) with a
    base index rule and a bound repair ("clip" or "midpoint"); `best` (the best
    row at the start of the generation, for the "best" rule) defaults to the
    argmin of `fit`."""
    pop = _f32(pop)
    fit = np.ascontiguousarray(fit, dtype=np.float64)
    N, D = pop.shape
    i0, i1 = (0, N) if rows is None else rows
    n = i1 - i0
    pop_out = np.empty_like(pop)
    fit_out = np.empty_like(fit)
    draws = np.empty((n, 5), dtype=np.int32)
    trial = np.empty((n, D), dtype=np.float32) if want_trial else None
    ftrial = np.empty(n, dtype=np.float64)
    accept = np.empty(n, dtype=np.uint8)
    msk = np.empty((n, D), dtype=np.uint8) if want_mask else None
    shift, rot = _f32(shift), _f32(rot)
    if best is None:
        best = argmin(fit)
    rc = lib().or_step_base(N, D, float(F), float(Cr), XO[xo], OBJ[obj] if isinstance(obj, str) else int(obj),
                            float(lo), float(hi), int(seed), int(inst), int(g), float(ackley_b),
                            _ptr(shift), _ptr(rot), _ptr(pop), _ptr(fit), _ptr(pop_out), _ptr(fit_out),
                            i0, i1, _ptr(draws), _ptr(trial), _ptr(ftrial), _ptr(accept), _ptr(msk),
                            BASE[base] if isinstance(base, str) else int(base), int(best),
                            REPAIR[repair] if isinstance(repair, str) else int(repair))
    if rc != 0:
        raise ValueError("oracle step rejected its arguments")
    return StepResult(pop_out, fit_out, draws, trial, ftrial, accept.astype(bool), msk)


def run(N, D, F, Cr, xo, obj, lo, hi, seed, G, inst=0, ackley_b=0.2, shift=None, rot=None,
        pop=None, base="distinct"):
    """Init (or take `pop`), evaluate, then G generations. Returns
    (pop, fit, best_index, best_f, best_gen, accepts, sumL)."""
    if pop is None:
        pop = init(N, D, lo, hi, seed, inst)
    fit = evaluate(obj, pop, ackley_b, shift, rot)
    b = argmin(fit)
    best_f, best_gen = fit[b], 0
    accepts = 0
    sumL = 0
    for g in range(G):
        s = step(pop, fit, F, Cr, xo, obj, lo, hi, seed, g, inst, ackley_b, shift, rot,
                 want_trial=False, base=base)
        pop, fit = s.pop, s.fit
        accepts += int(s.accept.sum())
        sumL += int(s.L.astype(np.int64).sum())
        b = argmin(fit)
        if fit[b] < best_f:
            best_f, best_gen = fit[b], g + 1
    return pop, fit, argmin(fit), best_f, best_gen, accepts, sumL
