"""GB300 (sm_103a) differential-evolution generation step (arXiv 2101.06599).

libde.so (csrc/, C ABI in include/de.h) runs the fused DE/rand/1 generation —
Philox draws, binomial / classic exponential / NEC crossover, mutation of
masked genes, clipping, FP32 fitness, greedy selection — on the GPU. This
package holds the build step, the ctypes binding (de.py) and the seeded
synthetic workloads (workloads.py).
"""
from .de import (Batch, DEError, Optimizer, de_batch_best, de_batch_create, de_batch_debug_step,
                 de_batch_autotune, de_batch_get_groups, de_batch_get_population, de_batch_set_groups,
                 de_batch_set_population, de_batch_size, de_batch_stats, de_best, de_best_async, de_create,
                 de_debug_step, de_destroy, de_get_kernel, de_get_pipeline, de_get_launch, de_get_population, de_load,
                 de_prepare_run, de_run, de_save, de_set_kernel, de_set_launch, de_set_pipeline, de_set_population,
                 de_stats, de_step, de_strerror, de_synchronize, de_version, load_library,
                 de_nec_step_noalloc, use_torch_allocator, best_record_bytes, parse_best_record)

__all__ = ["Batch", "DEError", "Optimizer", "de_batch_best", "de_batch_create", "de_batch_debug_step",
           "de_batch_autotune", "de_batch_get_groups", "de_batch_get_population", "de_batch_set_groups",
           "de_batch_set_population", "de_batch_size", "de_batch_stats", "de_best", "de_best_async", "de_create",
           "de_debug_step", "de_destroy", "de_get_kernel", "de_get_pipeline", "de_get_launch", "de_get_population",
           "de_load", "de_prepare_run", "de_run", "de_save", "de_set_kernel", "de_set_launch", "de_set_pipeline",
           "de_set_population", "de_stats", "de_step", "de_strerror", "de_synchronize", "de_version",
           "load_library", "de_nec_step_noalloc", "use_torch_allocator", "best_record_bytes", "parse_best_record"]
