"""The C-ABI library loads on a machine without a GPU, exports every call
include/*.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2101_06599_gb300 import build as B
from paper_2101_06599_gb300 import de as DE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(de_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return DE.load_library()


def test_header_declares_the_calls():
    names = declared_functions()
    for required in ("de_create", "de_step", "de_run", "de_best", "de_stats", "de_destroy",
                     "de_get_population", "de_set_population", "de_save", "de_load", "de_debug_step",
                     "de_batch_create", "de_batch_autotune", "de_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_version(lib):
    assert DE.de_strerror(0) == "ok"
    assert DE.de_strerror(DE.DE_EINVAL) == "invalid argument"
    assert DE.de_version() >= 100


@pytest.mark.parametrize("kw", [
    dict(N=3), dict(D=0), dict(D=40000), dict(CR=1.5), dict(CR=-0.1), dict(CR=float("nan")),
    dict(F=float("nan")), dict(F=float("inf")), dict(bounds=(1.0, 1.0)), dict(bounds=(2.0, -2.0)),
    dict(bounds=(float("-inf"), 0.0)), dict(xo=7), dict(obj=99),
])
def test_create_rejects_invalid_arguments(lib, kw):
    args = dict(N=16, D=8, F=0.5, CR=0.9, xo="nec", obj="sphere", bounds=(-1.0, 1.0), seed=1)
    args.update(kw)
    with pytest.raises(DE.DEError) as e:
        DE.de_create(**args)
    assert e.value.code == DE.DE_EINVAL


def test_rotated_objective_needs_shift_and_rotation(lib):
    with pytest.raises(DE.DEError) as e:
        DE.de_create(16, 8, 0.5, 0.9, "nec", "sr_rastrigin", (-100.0, 100.0), 1)
    assert e.value.code == DE.DE_EINVAL


@pytest.mark.parametrize("extra", [{"bound": 7}, {"margin_sigmas": -1.0}, {"margin_sigmas": float("nan")}])
def test_rotated_bound_parameters_are_validated(lib, extra):
    import numpy as np
    D = 8
    params = {"shift": np.zeros(D, np.float32), "rotation": np.eye(D, dtype=np.float32), "prec": "fp32"}
    params.update(extra)
    if "bound" in extra:
        DE.BOUND[7] = 7                      # an out-of-range enum value, passed through unchanged
        params["bound"] = 7
    try:
        with pytest.raises(DE.DEError) as e:
            DE.de_create(16, D, 0.5, 0.9, "nec", "sr_rastrigin", (-100.0, 100.0), 1, params=params)
        assert e.value.code == DE.DE_EINVAL
    finally:
        DE.BOUND.pop(7, None)


@pytest.mark.parametrize("args", [
    dict(ptr=0, ld=10, N=4, D=10, CR=0.5, xo=2),           # NULL output
    dict(ptr=64, ld=9, N=4, D=10, CR=0.5, xo=2),           # ld < D
    dict(ptr=64, ld=10, N=0, D=10, CR=0.5, xo=2),          # N < 1
    dict(ptr=64, ld=10, N=4, D=10, CR=1.5, xo=2),          # Cr outside [0, 1]
    dict(ptr=64, ld=10, N=4, D=10, CR=0.5, xo=7),          # no such crossover
])
def test_crossover_calls_validate_arguments(lib, args):
    import ctypes as C
    rc = lib.de_crossover_mask(C.c_void_p(args["ptr"]), args["ld"], args["N"], args["D"], args["CR"], args["xo"],
                               1, 0, 0, None)
    assert rc == DE.DE_EINVAL
    rc = lib.de_crossover_apply(C.c_void_p(args["ptr"]), C.c_void_p(128), C.c_void_p(256), args["ld"], args["N"],
                                args["D"], args["CR"], args["xo"], 1, 0, 0, None)
    assert rc == DE.DE_EINVAL


def test_crossover_apply_rejects_aliasing_and_bad_counters(lib):
    import ctypes as C
    p = C.c_void_p(64)
    assert lib.de_crossover_apply(p, p, C.c_void_p(128), 10, 4, 10, 0.5, 2, 1, 0, 0, None) == DE.DE_EINVAL
    assert lib.de_crossover_mask(p, 10, 4, 10, 0.5, 2, 1, -1, 0, None) == DE.DE_EINVAL       # generation < 0
    assert lib.de_crossover_mask(p, 10, 4, 10, 0.5, 2, 1, 0, 1 << 24, None) == DE.DE_EINVAL  # instance >= 2^24


def test_null_context_calls_are_rejected(lib):
    assert lib.de_step(None) == DE.DE_EINVAL
    assert lib.de_run(None, 3) == DE.DE_EINVAL
    assert lib.de_prepare_run(None, 3) == DE.DE_EINVAL
    assert lib.de_synchronize(None) == DE.DE_EINVAL
    assert lib.de_best(None, None, None, None, None) == DE.DE_EINVAL
    assert lib.de_batch_autotune(None, 3, None) == DE.DE_EINVAL
    assert lib.de_best_async(None, None) == DE.DE_EINVAL
    assert lib.de_batch_set_groups(None, None) == DE.DE_EINVAL
    lib.de_destroy(None)


def test_allocator_hook_must_be_paired(lib):
    assert lib.de_set_allocator(DE._alloc_cb, DE._FREE_FN(), None) == DE.DE_EINVAL
    assert lib.de_set_allocator(DE._ALLOC_FN(), DE._FREE_FN(), None) == DE.DE_OK


def test_create_without_a_device_fails_cleanly(lib):
    """On a machine without a GPU a valid request reaches allocation and
    fails there with a status code (exercises the whole host set-up path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(DE.DEError) as e:
        DE.de_create(64, 100, 0.5, 0.9, "nec", "sphere", (-1.0, 1.0), 1)
    assert e.value.code in (DE.DE_ENOMEM, DE.DE_ECUDA)
    specs = [dict(N=8, D=5, obj="sphere", bounds=(-1.0, 1.0)), dict(N=16, D=300, obj="ackley", bounds=(-30.0, 30.0))]
    with pytest.raises(DE.DEError) as e:
        DE.de_batch_create(specs, 1)
    assert e.value.code in (DE.DE_ENOMEM, DE.DE_ECUDA)


def test_best_record_size_matches_the_header():
    """de_best_async records: the header's size macro and the binding agree."""
    text = open(os.path.join(ROOT, "include", "de.h")).read()
    m = re.search(r"#define DE_BEST_RECORD_BYTES\(D\) \((\d+) \+ (\d+) \* \(size_t\)\(D\)\)", text)
    assert m, "DE_BEST_RECORD_BYTES not found"
    head, per = int(m.group(1)), int(m.group(2))
    for D in (1, 7, 1000):
        assert DE.best_record_bytes(D) == head + per * D
