"""Python binding of libde.so: the C ABI of include/de.h under the same names.

Argument marshalling only — every step of a generation runs in the CUDA
kernels of libde.so. PyTorch supplies device memory (the library's
allocator hook is routed to torch's caching allocator) and streams. There is
no CPU fallback: if libde.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DE_OK, DE_EINVAL, DE_ENOMEM, DE_ECUDA, DE_ETIMEOUT, DE_ESTATE, DE_EUNSUPPORTED = range(7)

XOVER = {"bin": 0, "exp": 1, "nec": 2}
OBJECTIVE = {"sphere": 0, "rastrigin": 1, "ackley": 2, "rosenbrock": 3, "griewank": 4,
             "elliptic": 5, "sr_rastrigin": 6, "sr_elliptic": 7}
PRECISION = {"fp32": 0, "tf32": 1, "bf16": 2, "fp16": 3}
BOUND = {"probabilistic": 0, "worst_case": 1}
BASE = {"distinct": 0, "random": 1, "offset": 2, "permutation": 3, "best": 4}
REPAIR = {"clip": 0, "midpoint": 1}


class DEError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, de_strerror(code), code))


class de_bounds(C.Structure):
    _fields_ = [("lo", C.c_float), ("hi", C.c_float)]


class de_objparams(C.Structure):
    _fields_ = [("ackley_b", C.c_double), ("shift", C.c_void_p), ("rotation", C.c_void_p),
                ("prec", C.c_int), ("incumbent_every", C.c_int32), ("bound", C.c_int),
                ("margin_sigmas", C.c_double), ("repair", C.c_int)]


class de_stats_t(C.Structure):
    _fields_ = [("generation", C.c_int64), ("accepts", C.c_uint64), ("masked_genes", C.c_uint64),
                ("reselected", C.c_uint64), ("best_gen", C.c_int64), ("best_f", C.c_double),
                ("best_index", C.c_int32), ("incumbent_f64", C.c_double), ("incumbent_gen", C.c_int64)]


class de_instance_spec(C.Structure):
    _fields_ = [("N", C.c_int32), ("D", C.c_int32), ("F", C.c_float), ("CR", C.c_double),
                ("xo", C.c_int), ("obj", C.c_int), ("b", de_bounds)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_live_blocks = {}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libde.so (building it first if asked). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libde.so not built (%s): run paper_2101_06599_gb300.build.build()" % path)
    L = C.CDLL(path)
    vp, i32, i64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double
    sig = {
        "de_version": ([], C.c_int),
        "de_strerror": ([C.c_int], C.c_char_p),
        "de_set_allocator": ([_ALLOC_FN, _FREE_FN, vp], C.c_int),
        "de_create": ([C.POINTER(vp), i32, i32, f32, f64, C.c_int, C.c_int, C.POINTER(de_objparams),
                       de_bounds, C.c_uint64, vp], C.c_int),
        "de_destroy": ([vp], None),
        "de_step": ([vp], C.c_int),
        "de_run": ([vp, i32], C.c_int),
        "de_prepare_run": ([vp, i32], C.c_int),
        "de_synchronize": ([vp], C.c_int),
        "de_best": ([vp, vp, C.POINTER(f64), C.POINTER(i32), C.POINTER(i64)], C.c_int),
        "de_best_async": ([vp, vp], C.c_int),
        "de_stats": ([vp, C.POINTER(de_stats_t)], C.c_int),
        "de_get_population": ([vp, vp, vp], C.c_int),
        "de_set_population": ([vp, vp, vp], C.c_int),
        "de_save": ([vp, vp, C.POINTER(C.c_size_t)], C.c_int),
        "de_load": ([vp, vp, C.c_size_t], C.c_int),
        "de_debug_step": ([vp, vp, vp, vp, vp], C.c_int),
        "de_debug_lengths": ([vp, i32, vp, i32, vp, vp, vp], C.c_int),
        "de_debug_mask": ([vp, i32, vp], C.c_int),
        "de_set_launch": ([vp, i32, i32], C.c_int),
        "de_set_wait_limit": ([vp, i64], C.c_int),
        "de_get_wait_limit": ([vp, C.POINTER(i64)], C.c_int),
        "de_get_launch": ([vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "de_set_kernel": ([vp, i32], C.c_int),
        "de_get_kernel": ([vp, C.POINTER(i32)], C.c_int),
        "de_set_pipeline": ([vp, i32, i32, i32], C.c_int),
        "de_get_pipeline": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "de_batch_create": ([C.POINTER(vp), i32, C.POINTER(de_instance_spec), C.c_uint64, vp], C.c_int),
        "de_batch_best": ([vp, i32, vp, C.POINTER(f64), C.POINTER(i32), C.POINTER(i64)], C.c_int),
        "de_batch_stats": ([vp, i32, C.POINTER(de_stats_t)], C.c_int),
        "de_batch_get_population": ([vp, i32, vp, vp], C.c_int),
        "de_batch_set_population": ([vp, i32, vp, vp], C.c_int),
        "de_batch_debug_step": ([vp, i32, vp, vp, vp, vp], C.c_int),
        "de_batch_set_groups": ([vp, C.POINTER(i32)], C.c_int),
        "de_batch_autotune": ([vp, i32, C.POINTER(i32)], C.c_int),
        "de_batch_get_groups": ([vp, C.POINTER(i32)], C.c_int),
        "de_batch_size": ([vp, C.POINTER(i32)], C.c_int),
        "de_nec_step_noalloc": ([vp, vp, vp, vp, i32, i32, i32, f32, f64, C.c_int, de_bounds, C.c_uint64,
                                 i64, vp], C.c_int),
        "de_set_base": ([vp, C.c_int], C.c_int),
        "de_get_base": ([vp, C.POINTER(C.c_int)], C.c_int),
        "de_crossover_mask": ([vp, i64, i32, i32, f64, C.c_int, C.c_uint64, i64, C.c_uint32, vp], C.c_int),
        "de_crossover_apply": ([vp, vp, vp, i64, i32, i32, f64, C.c_int, C.c_uint64, i64, C.c_uint32, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(code, where):
    if code != DE_OK:
        raise DEError(code, where)


def _host_ptr(a, dtype, size, writable):
    """Pointer to a contiguous host buffer (numpy array or CPU torch tensor)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous() or a.numel() < size:
            raise ValueError("host tensor must be a contiguous CPU tensor of %d elements" % size)
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous or a.size < size:
        raise ValueError("host array must be a C-contiguous %s array of %d elements" % (dtype, size))
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return C.c_void_p(a.ctypes.data)


# ---- allocator hook: torch's caching allocator --------------------------------
def _torch_alloc(nbytes, stream, user):
    import torch
    try:
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
    except RuntimeError:
        return None
    _live_blocks[t.data_ptr()] = t
    return t.data_ptr()


def _torch_free(ptr, nbytes, stream, user):
    _live_blocks.pop(ptr, None)


_alloc_cb = _ALLOC_FN(_torch_alloc)
_free_cb = _FREE_FN(_torch_free)


def use_torch_allocator(enable: bool = True):
    L = load_library()
    if enable:
        _check(L.de_set_allocator(_alloc_cb, _free_cb, None), "de_set_allocator")
    else:
        _check(L.de_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "de_set_allocator")


# ---- the C ABI, one wrapper per call -----------------------------------------
def de_version():
    return int(load_library().de_version())


def de_strerror(code):
    return load_library().de_strerror(int(code)).decode()


def de_create(N, D, F, CR, xo, obj, bounds, seed, params=None, stream=None):
    """Returns an opaque context handle (int). `stream` is a cudaStream_t value
    (e.g. torch.cuda.Stream().cuda_stream) or None for the legacy stream."""
    L = load_library()
    h = C.c_void_p()
    pp = None
    keep = []
    if params is not None:
        shift = params.get("shift")
        rot = params.get("rotation")
        if shift is not None:
            shift = np.ascontiguousarray(shift, dtype=np.float32)
            keep.append(shift)
        if rot is not None:
            rot = np.ascontiguousarray(rot, dtype=np.float32)
            keep.append(rot)
        pp = de_objparams(float(params.get("ackley_b", 0.0)),
                          shift.ctypes.data if shift is not None else None,
                          rot.ctypes.data if rot is not None else None,
                          PRECISION.get(params.get("prec", "fp32"), 0),
                          int(params.get("incumbent_every", 0)),
                          BOUND[params.get("bound", "probabilistic")],
                          float(params.get("margin_sigmas", 0.0)),
                          REPAIR[params.get("repair", "clip")])
    xo_i = XOVER[xo] if isinstance(xo, str) else int(xo)
    obj_i = OBJECTIVE[obj] if isinstance(obj, str) else int(obj)
    rc = L.de_create(C.byref(h), int(N), int(D), float(F), float(CR), xo_i, obj_i,
                     C.byref(pp) if pp is not None else None,
                     de_bounds(float(bounds[0]), float(bounds[1])), int(seed) & (2**64 - 1),
                     C.c_void_p(stream) if stream else None)
    _check(rc, "de_create")
    return h.value


def de_destroy(ctx):
    load_library().de_destroy(C.c_void_p(ctx))


def de_step(ctx):
    _check(load_library().de_step(C.c_void_p(ctx)), "de_step")


def de_run(ctx, generations):
    _check(load_library().de_run(C.c_void_p(ctx), int(generations)), "de_run")


def de_prepare_run(ctx, generations):
    _check(load_library().de_prepare_run(C.c_void_p(ctx), int(generations)), "de_prepare_run")


def de_synchronize(ctx):
    _check(load_library().de_synchronize(C.c_void_p(ctx)), "de_synchronize")


def de_best(ctx, x_out=None):
    """Returns (f, idx, best_gen); writes the best row into x_out (D floats) if given."""
    f, idx, bg = C.c_double(), C.c_int32(), C.c_int64()
    xp = None if x_out is None else _host_ptr(x_out, np.float32, 1, True)
    _check(load_library().de_best(C.c_void_p(ctx), xp, C.byref(f), C.byref(idx), C.byref(bg)), "de_best")
    return f.value, idx.value, bg.value


def best_record_bytes(D):
    """Bytes of one de_best_async record for rows of D genes."""
    return 32 + 4 * int(D)


def de_best_async(ctx, record, D):
    """Queue the best row and value into `record` (a page-locked uint8 host
    buffer of best_record_bytes(D) bytes); read it with parse_best_record
    after de_synchronize."""
    _check(load_library().de_best_async(C.c_void_p(ctx), _host_ptr(record, np.uint8, best_record_bytes(D), True)),
           "de_best_async")


def parse_best_record(record, D):
    """(f, idx, best_gen, x) of a completed de_best_async record; raises the
    device error the record carries."""
    b = record.numpy() if hasattr(record, "numpy") else np.asarray(record)
    b = b.view(np.uint8)
    err = int(b[20:24].view(np.int32)[0])
    if err:
        raise DEError(err, "de_best_async")
    f = float(b[0:8].view(np.float64)[0])
    gen = int(b[8:16].view(np.int64)[0])
    idx = int(b[16:20].view(np.int32)[0])
    x = b[32:32 + 4 * D].view(np.float32).copy()
    return f, idx, gen, x


def de_stats(ctx):
    s = de_stats_t()
    _check(load_library().de_stats(C.c_void_p(ctx), C.byref(s)), "de_stats")
    return {k: getattr(s, k) for k, _ in de_stats_t._fields_}


def de_get_population(ctx, pop_out, fit_out):
    _check(load_library().de_get_population(C.c_void_p(ctx), _host_ptr(pop_out, np.float32, 1, True),
                                            _host_ptr(fit_out, np.float32, 1, True)), "de_get_population")


def de_set_population(ctx, pop, fit=None):
    _check(load_library().de_set_population(C.c_void_p(ctx), _host_ptr(pop, np.float32, 1, False),
                                            _host_ptr(fit, np.float32, 1, False)), "de_set_population")


def de_save(ctx):
    L = load_library()
    n = C.c_size_t(0)
    _check(L.de_save(C.c_void_p(ctx), None, C.byref(n)), "de_save")
    buf = (C.c_ubyte * n.value)()
    _check(L.de_save(C.c_void_p(ctx), buf, C.byref(n)), "de_save")
    return bytes(buf[: n.value])


def de_load(ctx, blob):
    buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
    _check(load_library().de_load(C.c_void_p(ctx), buf, len(blob)), "de_load")


def de_debug_step(ctx, trial_out=None, ftrial_out=None, accept_out=None, draws_out=None):
    _check(load_library().de_debug_step(
        C.c_void_p(ctx), _host_ptr(trial_out, np.float32, 1, True), _host_ptr(ftrial_out, np.float32, 1, True),
        _host_ptr(accept_out, np.uint8, 1, True), _host_ptr(draws_out, np.int32, 1, True)), "de_debug_step")


def de_debug_lengths(ctx, words, inst=0):
    """Eq. (9)'s L (table in global and in shared memory) and Alg. 8's
    continuation flag for each given 32-bit word (see include/de.h)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    n = int(w.size)
    Lg = np.empty(n, dtype=np.int32)
    Ls = np.empty(n, dtype=np.int32)
    ec = np.empty(n, dtype=np.uint8)
    _check(load_library().de_debug_lengths(C.c_void_p(ctx), int(inst), C.c_void_p(w.ctypes.data), n,
                                           C.c_void_p(Lg.ctypes.data), C.c_void_p(Ls.ctypes.data),
                                           C.c_void_p(ec.ctypes.data)), "de_debug_lengths")
    return Lg, Ls, ec.astype(bool)


def de_debug_mask(ctx, N, D, inst=0):
    """The N x D crossover mask (uint8, 1 = from the mutant) of the next generation."""
    m = np.empty((N, D), dtype=np.uint8)
    _check(load_library().de_debug_mask(C.c_void_p(ctx), int(inst), C.c_void_p(m.ctypes.data)), "de_debug_mask")
    return m


def de_set_wait_limit(ctx, ns):
    _check(load_library().de_set_wait_limit(C.c_void_p(ctx), int(ns)), "de_set_wait_limit")


def de_get_wait_limit(ctx):
    v = C.c_int64()
    _check(load_library().de_get_wait_limit(C.c_void_p(ctx), C.byref(v)), "de_get_wait_limit")
    return v.value


def de_set_launch(ctx, threads, vec4):
    _check(load_library().de_set_launch(C.c_void_p(ctx), int(threads), int(vec4)), "de_set_launch")


def de_get_launch(ctx):
    t, v = C.c_int32(), C.c_int32()
    _check(load_library().de_get_launch(C.c_void_p(ctx), C.byref(t), C.byref(v)), "de_get_launch")
    return t.value, v.value


def de_set_kernel(ctx, kind):
    _check(load_library().de_set_kernel(C.c_void_p(ctx), int(kind)), "de_set_kernel")


def de_set_base(ctx, base):
    b = BASE[base] if isinstance(base, str) else int(base)
    _check(load_library().de_set_base(C.c_void_p(ctx), b), "de_set_base")


def de_get_base(ctx):
    b = C.c_int()
    _check(load_library().de_get_base(C.c_void_p(ctx), C.byref(b)), "de_get_base")
    return {v: k for k, v in BASE.items()}[b.value]


def de_get_kernel(ctx):
    k = C.c_int32()
    _check(load_library().de_get_kernel(C.c_void_p(ctx), C.byref(k)), "de_get_kernel")
    return k.value


def de_set_pipeline(ctx, consumer_threads, stages=0, ctas_per_sm=0):
    _check(load_library().de_set_pipeline(C.c_void_p(ctx), int(consumer_threads), int(stages),
                                          int(ctas_per_sm)), "de_set_pipeline")


def de_get_pipeline(ctx):
    """(consumer_threads, stages, span_floats, ctas_per_sm) of the pipelined kernel."""
    a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load_library().de_get_pipeline(C.c_void_p(ctx), C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
           "de_get_pipeline")
    return a.value, b.value, c.value, d.value


def de_batch_create(specs, seed, stream=None):
    L = load_library()
    arr = (de_instance_spec * len(specs))()
    for k, s in enumerate(specs):
        arr[k] = de_instance_spec(int(s["N"]), int(s["D"]), float(s.get("F", 0.5)), float(s.get("CR", 0.9)),
                                  XOVER[s.get("xo", "nec")], OBJECTIVE[s["obj"]],
                                  de_bounds(float(s["bounds"][0]), float(s["bounds"][1])))
    h = C.c_void_p()
    _check(L.de_batch_create(C.byref(h), len(specs), arr, int(seed), C.c_void_p(stream) if stream else None),
           "de_batch_create")
    return h.value


def de_batch_best(ctx, inst, x_out=None):
    f, idx, bg = C.c_double(), C.c_int32(), C.c_int64()
    xp = None if x_out is None else _host_ptr(x_out, np.float32, 1, True)
    _check(load_library().de_batch_best(C.c_void_p(ctx), int(inst), xp, C.byref(f), C.byref(idx), C.byref(bg)),
           "de_batch_best")
    return f.value, idx.value, bg.value


def de_batch_stats(ctx, inst):
    s = de_stats_t()
    _check(load_library().de_batch_stats(C.c_void_p(ctx), int(inst), C.byref(s)), "de_batch_stats")
    return {k: getattr(s, k) for k, _ in de_stats_t._fields_}


def de_batch_get_population(ctx, inst, pop_out, fit_out):
    _check(load_library().de_batch_get_population(C.c_void_p(ctx), int(inst), _host_ptr(pop_out, np.float32, 1, True),
                                                  _host_ptr(fit_out, np.float32, 1, True)),
           "de_batch_get_population")


def de_batch_set_population(ctx, inst, pop, fit=None):
    _check(load_library().de_batch_set_population(C.c_void_p(ctx), int(inst), _host_ptr(pop, np.float32, 1, False),
                                                  _host_ptr(fit, np.float32, 1, False)),
           "de_batch_set_population")


def de_batch_debug_step(ctx, inst, trial_out=None, ftrial_out=None, accept_out=None, draws_out=None):
    _check(load_library().de_batch_debug_step(
        C.c_void_p(ctx), int(inst), _host_ptr(trial_out, np.float32, 1, True),
        _host_ptr(ftrial_out, np.float32, 1, True), _host_ptr(accept_out, np.uint8, 1, True),
        _host_ptr(draws_out, np.int32, 1, True)), "de_batch_debug_step")


def de_batch_size(ctx):
    n = C.c_int32()
    _check(load_library().de_batch_size(C.c_void_p(ctx), C.byref(n)), "de_batch_size")
    return n.value


def de_batch_autotune(ctx, reps, n_inst):
    out = (C.c_int32 * n_inst)()
    _check(load_library().de_batch_autotune(C.c_void_p(ctx), int(reps), out), "de_batch_autotune")
    return [int(v) for v in out]


def de_batch_set_groups(ctx, groups):
    arr = (C.c_int32 * len(groups))(*[int(g) for g in groups])
    _check(load_library().de_batch_set_groups(C.c_void_p(ctx), arr), "de_batch_set_groups")


def de_batch_get_groups(ctx):
    n = de_batch_size(ctx)
    arr = (C.c_int32 * n)()
    _check(load_library().de_batch_get_groups(C.c_void_p(ctx), arr), "de_batch_get_groups")
    return [int(v) for v in arr]


def de_nec_step_noalloc(pop_in, fit_in, pop_out, fit_out, N, D, pitch, F, CR, obj, bounds, seed,
                        generation, stream=None):
    """One NEC generation on caller-owned device buffers (addresses as ints);
    the library allocates nothing for it. See include/de.h."""
    obj_i = OBJECTIVE[obj] if isinstance(obj, str) else int(obj)
    _check(load_library().de_nec_step_noalloc(
        C.c_void_p(pop_in), C.c_void_p(fit_in), C.c_void_p(pop_out), C.c_void_p(fit_out), int(N), int(D),
        int(pitch), float(F), float(CR), obj_i, de_bounds(float(bounds[0]), float(bounds[1])),
        int(seed) & (2**64 - 1), int(generation), C.c_void_p(stream) if stream else None),
        "de_nec_step_noalloc")


class Batch:
    """Many independent DE instances on the current CUDA device, advanced
    together (de_batch_create / de_step / de_run / de_batch_best ...).

    specs: list of dicts with N, D, obj, bounds and optionally F, CR, xo."""

    def __init__(self, specs, seed=1, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libde needs a CUDA GPU; no CPU fallback exists")
        use_torch_allocator(True)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.specs = [dict(s) for s in specs]
        self.ctx = de_batch_create(self.specs, seed, self.stream.cuda_stream)

    def __len__(self):
        return len(self.specs)

    def step(self):
        de_step(self.ctx)

    def run(self, generations):
        de_run(self.ctx, generations)

    def prepare_run(self, generations):
        """Build the graph that run(generations) replays, without running it."""
        de_prepare_run(self.ctx, generations)

    def synchronize(self):
        de_synchronize(self.ctx)

    def stats(self, inst=None):
        return de_stats(self.ctx) if inst is None else de_batch_stats(self.ctx, inst)

    def best(self, inst):
        x = np.empty(self.specs[inst]["D"], dtype=np.float32)
        f, idx, bg = de_batch_best(self.ctx, inst, x)
        return x, f, idx, bg

    def population(self, inst):
        N, D = self.specs[inst]["N"], self.specs[inst]["D"]
        pop = np.empty((N, D), dtype=np.float32)
        fit = np.empty(N, dtype=np.float32)
        de_batch_get_population(self.ctx, inst, pop, fit)
        return pop, fit

    def set_population(self, inst, pop, fit=None):
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        if fit is not None:
            fit = np.ascontiguousarray(fit, dtype=np.float32)
        de_batch_set_population(self.ctx, inst, pop, fit)

    def debug_step(self, inst):
        N, D = self.specs[inst]["N"], self.specs[inst]["D"]
        trial = np.empty((N, D), dtype=np.float32)
        ft = np.empty(N, dtype=np.float32)
        acc = np.empty(N, dtype=np.uint8)
        dr = np.empty((N, 5), dtype=np.int32)
        de_batch_debug_step(self.ctx, inst, trial, ft, acc, dr)
        return trial, ft, acc.astype(bool), dr

    def set_base(self, base):
        de_set_base(self.ctx, base)

    def debug_lengths(self, inst, words):
        return de_debug_lengths(self.ctx, words, inst)

    def debug_mask(self, inst):
        return de_debug_mask(self.ctx, self.specs[inst]["N"], self.specs[inst]["D"], inst)

    def set_wait_limit(self, ns):
        de_set_wait_limit(self.ctx, ns)

    def wait_limit(self):
        return de_get_wait_limit(self.ctx)

    def groups(self):
        return de_batch_get_groups(self.ctx)

    def set_groups(self, groups):
        de_batch_set_groups(self.ctx, groups)

    def autotune(self, reps=5):
        """Time the candidate row kernels per group of instances and keep the
        fastest (results do not depend on the choice); returns the groups."""
        return de_batch_autotune(self.ctx, reps, len(self.specs))

    def close(self):
        if getattr(self, "ctx", None):
            de_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience object --------------------------------------------------------
class Optimizer:
    """One DE population on the current CUDA device, on its own torch stream.

    Wraps de_create / de_step / de_run / de_best / de_stats / ... of libde.so.
    """

    def __init__(self, N, D, F=0.5, CR=0.9, xo="nec", obj="sphere", bounds=(-100.0, 100.0), seed=1,
                 params=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libde needs a CUDA GPU; no CPU fallback exists")
        use_torch_allocator(True)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.N, self.D = int(N), int(D)
        self.ctx = de_create(N, D, F, CR, xo, obj, bounds, seed, params, self.stream.cuda_stream)

    def step(self):
        de_step(self.ctx)

    def run(self, generations):
        de_run(self.ctx, generations)

    def prepare_run(self, generations):
        """Build the graph that run(generations) replays, without running it."""
        de_prepare_run(self.ctx, generations)

    def synchronize(self):
        de_synchronize(self.ctx)

    def best(self):
        x = np.empty(self.D, dtype=np.float32)
        f, idx, bg = de_best(self.ctx, x)
        return x, f, idx, bg

    def stats(self):
        return de_stats(self.ctx)

    def population(self):
        pop = np.empty((self.N, self.D), dtype=np.float32)
        fit = np.empty(self.N, dtype=np.float32)
        de_get_population(self.ctx, pop, fit)
        return pop, fit

    def set_population(self, pop, fit=None):
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        if fit is not None:
            fit = np.ascontiguousarray(fit, dtype=np.float32)
        de_set_population(self.ctx, pop, fit)

    def debug_step(self):
        trial = np.empty((self.N, self.D), dtype=np.float32)
        ft = np.empty(self.N, dtype=np.float32)
        acc = np.empty(self.N, dtype=np.uint8)
        dr = np.empty((self.N, 5), dtype=np.int32)
        de_debug_step(self.ctx, trial, ft, acc, dr)
        return trial, ft, acc.astype(bool), dr

    def debug_lengths(self, words):
        return de_debug_lengths(self.ctx, words, 0)

    def debug_mask(self):
        return de_debug_mask(self.ctx, self.N, self.D, 0)

    def save(self):
        return de_save(self.ctx)

    def load(self, blob):
        de_load(self.ctx, blob)

    def set_launch(self, threads, vec4):
        de_set_launch(self.ctx, threads, vec4)

    def launch(self):
        return de_get_launch(self.ctx)

    def set_base(self, base):
        """Base index rule: "distinct" (default), "random", "offset",
        "permutation" or "best" (see de_set_base)."""
        de_set_base(self.ctx, base)

    def base(self):
        return de_get_base(self.ctx)

    def set_kernel(self, kind):
        de_set_kernel(self.ctx, kind)

    def kernel(self):
        return de_get_kernel(self.ctx)

    def set_pipeline(self, consumer_threads, stages=0, ctas_per_sm=0):
        de_set_pipeline(self.ctx, consumer_threads, stages, ctas_per_sm)

    def pipeline(self):
        return de_get_pipeline(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            de_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def de_crossover_mask(mask, ld, N, D, CR, xo, seed, generation, instance=0, stream=None):
    """The N x D crossover mask of generation `generation` (1 = the gene
    crosses) into device bytes at `mask` (rows of `ld` bytes), the draws of
    de_step. See include/de.h."""
    xo_i = XOVER[xo] if isinstance(xo, str) else int(xo)
    _check(load_library().de_crossover_mask(
        C.c_void_p(mask), int(ld), int(N), int(D), float(CR), xo_i, int(seed) & (2**64 - 1), int(generation),
        int(instance), C.c_void_p(stream) if stream else None), "de_crossover_mask")


def de_crossover_apply(u, x, v, ld, N, D, CR, xo, seed, generation, instance=0, stream=None):
    """U = mask ? V : X on device matrices (rows of `ld` floats), the mask of
    de_crossover_mask. See include/de.h."""
    xo_i = XOVER[xo] if isinstance(xo, str) else int(xo)
    _check(load_library().de_crossover_apply(
        C.c_void_p(u), C.c_void_p(x), C.c_void_p(v), int(ld), int(N), int(D), float(CR), xo_i,
        int(seed) & (2**64 - 1), int(generation), int(instance), C.c_void_p(stream) if stream else None),
        "de_crossover_apply")
