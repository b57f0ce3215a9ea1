/*
 * de.h — C ABI of the GB300 (sm_103a) differential-evolution generation
 * library (libde.so).
 *
 * The method is DE/rand/1 as parallelised in Pan, "Performance Analysis and
 * Improvement of Parallel Differential Evolution" (arXiv 2101.06599):
 * one generation = donor draws, crossover mask (binomial, Eq. 2 / Alg. 7;
 * classic exponential, Alg. 8; new exponential crossover NEC, Eq. 9 with
 * Alg. 9 / Alg. 10), differential mutation on the masked genes (Eq. 1),
 * bound repair, evaluation of the whole trial population, and greedy
 * selection (Alg. 2). The calls follow the paper's statement of the problem:
 * parameters Cr, F, Np and a stop criterion (Alg. 1 / Alg. 2, first line),
 * evaluation as its own stage (Section 2, before Alg. 2), best value and best
 * generation as outputs (Tables III-V).
 *
 * Conventions for every call:
 *  - Return value: DE_OK (0) or a positive de_status code; nothing calls
 *    exit/abort and no kernel traps. de_strerror() names a code.
 *  - Host pointers are caller-owned, read or written during the call only,
 *    never retained. Host arrays are dense row-major (row length D floats).
 *  - Device memory is owned by the context, obtained from the allocator set
 *    with de_set_allocator (cudaMalloc if none), and released by
 *    de_destroy.
 *  - Work is queued on the CUDA stream given to de_create (NULL = legacy
 *    default stream). de_step/de_run only enqueue; errors raised by queued
 *    work surface at the next call that synchronises (de_best, de_stats,
 *    de_get_population, de_save, de_synchronize) as DE_ECUDA.
 *  - Every wait inside a kernel is bounded. A wait that gives up records
 *    DE_ETIMEOUT in the context's device state; de_synchronize, de_stats and
 *    de_best (and their batched forms) report it. From the first call that
 *    reports a device error on, the context refuses to launch generations:
 *    de_step, de_run and the debug steps return DE_ESTATE. Populations can
 *    still be read; de_destroy releases the context as usual.
 *  - A context is not thread-safe; use one host thread per context.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key (seed low
 * word, seed high word) and counter (block, row, generation, stream<<24 |
 * instance). Every draw is a pure function of (seed, instance, generation,
 * row), so draws do not depend on the launch shape, and de_save/de_load
 * resume bit-identically. FP32 fitness sums are reduced in a fixed order
 * set by the launch shape (de_set_launch), so a run is deterministic for a
 * given shape.
 */
#ifndef DE_H
#define DE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef enum {
  DE_OK = 0,
  DE_EINVAL = 1,       /* invalid argument (see each call)                   */
  DE_ENOMEM = 2,       /* device or host allocation failed                   */
  DE_ECUDA = 3,        /* a CUDA runtime call or queued kernel failed        */
  DE_ETIMEOUT = 4,     /* a bounded device-side wait gave up                 */
  DE_ESTATE = 5,       /* call not valid for this context's state            */
  DE_EUNSUPPORTED = 6  /* valid request this build does not implement        */
} de_status;

/* ---- crossover (Section 3) -------------------------------------------- */
typedef enum {
  DE_XOVER_BIN = 0,    /* binomial: gene j crosses iff rand < Cr or j = j_rand (Eq. 2, Alg. 7) */
  DE_XOVER_EXP = 1,    /* classic exponential: sequential walk from j_rand (Alg. 8)            */
  DE_XOVER_NEC = 2     /* new exponential: L from Eq. (9), genes ((j - j_rand) mod D) < L       */
} de_crossover;

/* ---- objectives -------------------------------------------------------- */
typedef enum {
  DE_OBJ_SPHERE = 0,        /* sum x^2                                            */
  DE_OBJ_RASTRIGIN = 1,     /* 10 D + sum (x^2 - 10 cos 2 pi x)                   */
  DE_OBJ_ACKLEY = 2,        /* Section 4; inner constant b (de_objparams)          */
  DE_OBJ_ROSENBROCK = 3,    /* Section 4: sum_{j<D-1} 100 (x_j^2 - x_{j+1})^2 + (1 - x_j)^2 */
  DE_OBJ_GRIEWANK = 4,      /* Section 4: sum x^2 / 4000 - prod cos(x_j / sqrt j) + 1 */
  DE_OBJ_ELLIPTIC = 5,      /* sum 10^(6 j / (D-1)) x_j^2, j = 0 .. D-1            */
  DE_OBJ_SR_RASTRIGIN = 6,  /* Rastrigin of z = R (x - o)                          */
  DE_OBJ_SR_ELLIPTIC = 7    /* elliptic of z = R (x - o)                           */
} de_objective;

/* Precision of the z = R (x - o) product of the shifted-rotated objectives.
 * FP32: SIMT FMA chains. BF16 and FP16: tensor-core products of split
 * operands (a = a_hi + a_lo, R = R_hi + R_lo, three products), FP32
 * accumulation, selections made certain by an error bound and the rest
 * re-evaluated in FP32, so every decision is the FP32 path's. BF16 splits
 * carry 16 bits of each operand; FP16 splits carry 22, scaled by powers of
 * two (x - o by 2^s with max |x - o| 2^s below 2^15 from the box, R by 2^14
 * over its largest entry) so that both halves stay normal, which makes the
 * bound about 60 % narrower and sends fewer rows to the re-evaluation; the
 * halves of components below ~2^-11 of the box's reach lose bits to FP16's
 * subnormal range, which the bound counts. Both need D a multiple of 256 and
 * a GB300 (sm_103); TF32 returns DE_EUNSUPPORTED. */
typedef enum { DE_PREC_FP32 = 0, DE_PREC_TF32 = 1, DE_PREC_BF16 = 2, DE_PREC_FP16 = 3 } de_precision;

/* Error bound that decides which BF16- or FP16-path selections are certain
 * (the rest are re-evaluated with the FP32 product, so that decisions match
 * the FP32 path). PROBABILISTIC: margin_sigmas standard deviations of |f_BF16 -
 * f_FP32| under the standard model of independent, zero-mean rounding errors
 * (Hoeffding's inequality), with the accumulation's partial sums taken as at
 * most 4 |x - o|_2 / sqrt(D) (rotations with delocalised rows, such as a
 * random orthogonal R). WORST_CASE: the deterministic bound, valid for any R,
 * which at D ~ 1000 sends almost every row to the FP32 re-evaluation. */
typedef enum { DE_BOUND_PROBABILISTIC = 0, DE_BOUND_WORST_CASE = 1 } de_bound_kind;

/* Search box, the same for every dimension (Section 4 gives one interval
 * per function). Requires lo < hi, both finite. Mutant genes outside it are
 * repaired (de_repair; the paper names no rule). */
typedef struct { float lo, hi; } de_bounds;

/* Bound repair of a mutant gene v outside [lo, hi], the paper being silent:
 * CLIP sets it to the violated bound; MIDPOINT to the midpoint between the
 * violated bound and the target (parent) gene x of the same row and column,
 * fl(fl(bound + x) 0.5) in FP32, which lies in the box because x does. Only
 * genes the crossover takes from the mutant are repaired. */
typedef enum { DE_REPAIR_CLIP = 0, DE_REPAIR_MIDPOINT = 1 } de_repair;

/* Optional objective parameters; pass NULL for the defaults. */
typedef struct {
  double ackley_b;          /* Ackley inner constant; 0 selects 0.2 (Section 4 prints 0.02) */
  const float *shift;       /* host, D floats: o of the shifted-rotated objectives (copied) */
  const float *rotation;    /* host, D*D floats, row-major R (copied)                       */
  de_precision prec;        /* shifted-rotated objectives: product precision                */
  int32_t incumbent_every;  /* shifted-rotated: FP64 re-evaluation of the best every K
                               generations (0 selects 50)                                  */
  de_bound_kind bound;      /* BF16/FP16 product: which error bound decides certain selections */
  double margin_sigmas;     /* PROBABILISTIC bound: margin in standard deviations (0 selects
                               8; the model's failure probability per decision is at most
                               2 exp(-m^2 / 2))                                             */
  de_repair repair;         /* bound repair (CLIP when zero); batched instances always clip  */
} de_objparams;

/* Counters kept on the device and read by de_stats. */
typedef struct {
  int64_t generation;       /* generations completed                                     */
  uint64_t accepts;         /* trials that replaced their parent, summed over generations */
  uint64_t masked_genes;    /* genes taken from the mutant: sum of L (exp, NEC) or of the
                               mask popcount (bin), summed over generations               */
  uint64_t reselected;      /* shifted-rotated, low precision: rows re-evaluated in FP32  */
  int64_t best_gen;         /* generation at which the best value last strictly improved  */
  double best_f;            /* best fitness (FP32 value, widened)                          */
  int32_t best_index;       /* row holding it; lowest index on ties                       */
  double incumbent_f64;     /* shifted-rotated: the best row's objective recomputed in FP64
                               every incumbent_every generations (0 when incumbent_gen is -1) */
  int64_t incumbent_gen;    /* generation of that re-evaluation (-1 = none)                */
} de_stats_t;

typedef struct de_ctx de_ctx;

/* ---- device memory ----------------------------------------------------- */
/* Allocator used by every later de_create / de_batch_create. alloc returns a
 * device pointer of at least `bytes` bytes aligned to 256 bytes, or NULL;
 * free releases it. `stream` is the context's stream. Pass NULL, NULL to go
 * back to cudaMalloc/cudaFree. Process-wide; not thread-safe. */
typedef void *(*de_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*de_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int de_set_allocator(de_alloc_fn alloc, de_free_fn free_fn, void *user);

/* ---- lifecycle --------------------------------------------------------- */
/* Create a population of N individuals with D genes (Alg. 2, first lines):
 * x_ij = clip(lo + (hi - lo) * u_ij) with u_ij = (w >> 8) * 2^-24 from
 * Philox stream 0, then evaluate every row (the call returns after this
 * set-up has finished on the device).
 *   N >= 4 (three distinct donors other than i), N < 2^31 / 4;
 *   1 <= D <= 32768; N * D < 2^40;
 *   F finite; CR in [0, 1]; xo and obj valid enum values;
 *   shifted-rotated objectives need p->shift and p->rotation.
 * Errors: DE_EINVAL, DE_ENOMEM, DE_ECUDA, DE_EUNSUPPORTED. */
int de_create(de_ctx **out, int32_t N, int32_t D, float F, double CR,
              de_crossover xo, de_objective obj, const de_objparams *p,
              de_bounds b, uint64_t seed, void *cuda_stream);

/* Release every buffer of the context (synchronises its stream). NULL is a no-op. */
void de_destroy(de_ctx *ctx);

/* ---- generations (Alg. 2, loop body) ----------------------------------- */
/* Enqueue one generation: draws, crossover, mutation of masked genes, clip,
 * evaluation of every trial (FP32), strict '<' selection, best tracking. */
int de_step(de_ctx *ctx);

/* Enqueue `generations` (>= 0) generations. Runs of 2 or more on a context
 * with its own stream are captured once per distinct count into a CUDA graph
 * (on the first run of that count, or by de_prepare_run) and replayed; a
 * setter that changes the launch (kernel, launch shape, pipeline, base rule,
 * wait limit) drops the cached graphs. */
int de_run(de_ctx *ctx, int32_t generations);

/* Capture and instantiate the graph that de_run(ctx, generations) replays,
 * without launching it: the population, fitness, best and generation count
 * are unchanged, and a later de_run of the same count only launches the
 * graph. A no-op returning DE_OK for counts below 2 and for a context on the
 * legacy (NULL) stream, whose runs are not captured. DE_EINVAL for a NULL
 * context or a negative count, DE_ESTATE for a failed context, DE_ECUDA if
 * the capture or the instantiation fails. */
int de_prepare_run(de_ctx *ctx, int32_t generations);

/* Block until the context's stream is idle; DE_ECUDA if queued work failed,
 * the device error code (DE_ETIMEOUT) if a kernel recorded one. */
int de_synchronize(de_ctx *ctx);

/* Limit, in nanoseconds of the GPU's global timer, of the device waits that
 * guard no copy or tensor-core operation in flight: the grid barrier of the
 * batched one-launch generation between its row plans and its rows. ns = 0
 * restores the default (1 s); DE_EINVAL for ns < 0. A CTA whose barrier wait
 * gives up records DE_ETIMEOUT and takes no rows; the CTAs the barrier
 * released process every row between them, so the generation is still
 * complete and identical to one without the timeout. The waits of the
 * pipelined and tensor-core kernels, which guard bulk copies and MMAs in
 * flight, keep their fixed 1 s limit. de_get_wait_limit reports the limit
 * in force. Drops the context's captured graphs. */
int de_set_wait_limit(de_ctx *ctx, int64_t ns);
int de_get_wait_limit(de_ctx *ctx, int64_t *ns);

/* ---- results ----------------------------------------------------------- */
/* Best individual so far (synchronises). Any output pointer may be NULL.
 * x_out: host, D floats. f_out: its fitness. idx_out: its row (lowest index
 * on ties). best_gen_out: generation of the last strict improvement (0 =
 * the initial population). */
int de_best(de_ctx *ctx, float *x_out, double *f_out, int32_t *idx_out,
            int64_t *best_gen_out);

/* Best individual so far, without waiting: queues on the context's stream
 * the gather of the best row and its copy into `record_out`, a host buffer
 * of DE_BEST_RECORD_BYTES(D) bytes that the caller owns (page-locked, or the
 * copy is staged and the call may block); the record is complete once the
 * stream has reached this point (de_synchronize). Layout: double best_f at
 * byte 0, int64 best_gen at 8, int32 best row at 16, int32 device error at
 * 20 (0 = none; else the code de_best would return), then the D floats of
 * the row at byte 32. Successive calls may target different records (a ring
 * of per-step results). DE_ESTATE on a batch. */
#define DE_BEST_RECORD_BYTES(D) (32 + 4 * (size_t)(D))
int de_best_async(de_ctx *ctx, void *record_out);

/* Device counters (synchronises). */
int de_stats(de_ctx *ctx, de_stats_t *out);

/* Copy the population (host N x D floats) and fitness (host N floats) out;
 * either may be NULL (synchronises). */
int de_get_population(de_ctx *ctx, float *pop_out, float *fit_out);

/* Replace the population with host N x D floats. fit = NULL evaluates every
 * row on the device; otherwise N host floats are taken as given. The best
 * is recomputed and best_gen set to the current generation. Genes are taken
 * as given (not clipped). Synchronises. */
int de_set_population(de_ctx *ctx, const float *pop, const float *fit);

/* ---- checkpoint / resume ----------------------------------------------- */
/* Serialise the whole state (parameters, generation, counters, best,
 * population, fitness; for a shifted-rotated context with a BF16 or FP16
 * product also the error bounds of the stored fitness values). With buf =
 * NULL, *len receives the size needed; otherwise *len must be at least that
 * and receives the bytes written. Synchronises. */
int de_save(de_ctx *ctx, void *buf, size_t *len);

/* Restore a state saved by de_save into a context created with the same N,
 * D, F, CR, crossover, objective, bounds and seed (DE_EINVAL otherwise).
 * The resumed run is bit-identical to an uninterrupted one. */
int de_load(de_ctx *ctx, const void *buf, size_t len);

/* ---- test hook ----------------------------------------------------------- */
/* Run one generation exactly like de_step and also report, per row, the
 * trial vector (host N x D floats), its FP32 fitness (N floats), the
 * selection decision (N bytes, 1 = accepted) and the draws (N x 5 int32:
 * r1, r2, r3, j_rand, L where L is the segment length for exp/NEC and the
 * mask popcount for bin). Any output may be NULL. Synchronises. */
int de_debug_step(de_ctx *ctx, float *trial_out, float *ftrial_out,
                  uint8_t *accept_out, int32_t *draws_out);

/* Test hook for the draws of Eq. (9) and Alg. 8 at given random words.
 * For each of the n words w[k] (host array; w / 2^32 is the uniform U of the
 * row), with the Cr, D and NEC threshold table of the context (instance
 * `inst` of a batch; 0 for a single population):
 *   L_global[k]  NEC's segment length L = min(ceil(ln U / ln Cr), D), Eq. (9)
 *                read exactly as L = smallest n >= 1 with Cr^n <= U (Cr^n the
 *                FP64 product Cr * Cr * ... rounded at each step), capped at D;
 *                U = 0 gives D, Cr = 0 gives 1, Cr = 1 gives D. Computed by the
 *                lookup the generation kernels use, on the table in global memory;
 *   L_shared[k]  the same through the copy of the table in shared memory that
 *                the pipelined kernel and the batched plans use (when the
 *                table has at most 4096 entries; else as L_global, as those
 *                kernels then do);
 *   exp_continue[k]  1 iff Alg. 8's walk continues on this word: U < Cr.
 * Outputs are host arrays of n elements; any may be NULL. Synchronises.
 * DE_EINVAL for n < 0, a NULL `words` with n > 0 or an invalid `inst`. */
int de_debug_lengths(de_ctx *ctx, int32_t inst, const uint32_t *words, int32_t n,
                     int32_t *L_global, int32_t *L_shared, uint8_t *exp_continue);

/* Test hook: the crossover mask (Eq. 2, Alg. 8, Alg. 9) that the next
 * generation of the context (instance `inst` of a batch; 0 for a single
 * population) uses: mask_out (host, N x D bytes, row-major) gets 1 where
 * gene j of row i is taken from the mutant, 0 where it is the parent's.
 * Computed by the draw functions of the generation kernels (j_rand from the
 * row's IDX block under the base rule in force, L from Eq. (9) or Alg. 8,
 * the binomial words from the row's BIN blocks); the population is not
 * touched. Synchronises. DE_EINVAL for a NULL mask_out or an invalid inst. */
int de_debug_mask(de_ctx *ctx, int32_t inst, uint8_t *mask_out);

/* ---- batched instances --------------------------------------------------- */
/* One independent DE problem of a batch. */
typedef struct {
  int32_t N, D;
  float F;
  double CR;
  de_crossover xo;
  de_objective obj;          /* non-rotated objectives only */
  de_bounds b;
} de_instance_spec;

/* Create a context running n_inst independent instances (1 <= n_inst <=
 * 2^24); instance k draws from Philox instance field k, so instance k of a
 * batch reproduces a single population whose draws use instance field k.
 * Each instance keeps its own population, fitness, counters and best. One
 * de_step / de_run step advances every instance by one generation: one
 * cooperative kernel launch (draws, rows, close) when every instance is on
 * the staged kernel (the default for exp / NEC rows of D <= 2048), else a
 * few launches over all instances (draws, row kernels, close). The rows of
 * each instance are cut into spans of up to 32 rows (taken by warps from a
 * queue) or, for D > 2048, into tiles of 256 / G rows; the row kernel of
 * each instance is set by de_batch_set_groups or de_batch_autotune. A device
 * wait that gives up (1 s) is reported as DE_ETIMEOUT by the next
 * synchronising call. Per-instance limits as de_create
 * with D <= 16384 and non-rotated objectives (Ackley constant 0.2). The
 * initial populations are drawn and evaluated before the call returns.
 * Single-population calls (de_best, de_get_population, de_set_population,
 * de_debug_step, de_set_kernel, ...) return DE_ESTATE on a batch; de_save
 * and de_load return DE_EUNSUPPORTED. de_stats returns totals: summed
 * accepts and masked genes, the common generation, and in best_f / best_gen
 * / best_index the best value over all instances, its generation and the
 * instance that holds it. */
int de_batch_create(de_ctx **out, int32_t n_inst, const de_instance_spec *specs,
                    uint64_t seed, void *cuda_stream);

/* Best of instance `inst` (synchronises); outputs as de_best, x_out has the
 * instance's D floats. */
int de_batch_best(de_ctx *ctx, int32_t inst, float *x_out, double *f_out,
                  int32_t *idx_out, int64_t *best_gen_out);

/* Counters of instance `inst`, as de_stats for a single population. */
int de_batch_stats(de_ctx *ctx, int32_t inst, de_stats_t *out);

/* Population I/O of instance `inst`, as de_get_population /
 * de_set_population (host arrays of N_inst x D_inst floats). */
int de_batch_get_population(de_ctx *ctx, int32_t inst, float *pop_out, float *fit_out);
int de_batch_set_population(de_ctx *ctx, int32_t inst, const float *pop, const float *fit);

/* Test hook: one generation of every instance, reporting for instance
 * `inst` what de_debug_step reports for a single population. */
int de_batch_debug_step(de_ctx *ctx, int32_t inst, float *trial_out, float *ftrial_out,
                        uint8_t *accept_out, int32_t *draws_out);

/* Row kernel per instance (one value per instance):
 *   -G         the staged warp pipeline (exp and NEC only, D <= 2048) with G
 *              lanes per row (G = 4, 8, 16 or 32): each warp loads the next
 *              pass of up to 32 rows / 8 KB into registers while it
 *              processes the previous one from shared memory;
 *   1          the staged pipeline with its default G (32);
 *   2          the streaming kernel (exp and NEC only, any D): one warp per
 *              row, the row read in chunks of 512 genes straight into
 *              registers while the previous chunk is processed;
 *   G = 4..256 (a power of two with ceil(ceil(D/4) / G) <= 16) register
 *              tiles of G threads per row (one warp of 32 / G rows for
 *              G <= 32, a CTA of 256 / G rows above);
 *   0          the default: 1 for exp and NEC rows of D <= 2048, else the
 *              smallest such G.
 * de_batch_get_groups reports staged instances as -G. Draws are unchanged by
 * the choice, and so are fitness values, selections and trajectories for
 * every choice with at most 32 threads per row (staged, streaming, and
 * G = 4..32): those kernels sum the FP32 fitness in one fixed order. G > 32 (needed only
 * for D > 2048) sums in another order. Returns DE_EINVAL for an invalid
 * value; the context is unchanged then. */
int de_batch_set_groups(de_ctx *ctx, const int32_t *groups);
int de_batch_get_groups(de_ctx *ctx, int32_t *groups);

/* Autotuner: pick each instance's row kernel (the values above) by timing.
 * Instances are grouped by crossover and the octave of ceil(D/4) (rows of
 * D <= 2048; wider rows keep their tiles). For each group in turn, every
 * candidate (register tiles of 4..32 lanes per row; for exp and NEC the
 * staged pipeline with 4..32 lanes) is timed over `reps` (1..1000) runs of
 * the row kernels of one generation of every instance, the other groups as
 * they stand, so that kernels which slow each other down when they run
 * together (instruction cache, occupancy) are judged together; the fastest
 * is kept. The trials reuse the draws of the current generation and leave
 * populations, fitness, counters and the generation as they were, and the choice changes no result (every
 * candidate sums the fitness in one order). Synchronises; drops captured
 * graphs. groups_out (n_inst values, may be NULL) receives the choice as
 * de_batch_get_groups reports it. DE_ESTATE on a single population. */
int de_batch_autotune(de_ctx *ctx, int32_t reps, int32_t *groups_out);
/* Number of instances (0 for a single-population context). */
int de_batch_size(de_ctx *ctx, int32_t *n_inst);

/* ---- launch shape --------------------------------------------------------- */
/* Each row is processed by one CTA of `threads` threads (multiple of 32,
 * <= 512), each holding `vec4` float4 slots of the row in registers (vec4 in
 * {1, 2, 4, 8, 16}); threads * vec4 * 4 must cover D. de_create picks a
 * shape; this overrides it (tuning only: draws are unchanged, FP32 fitness
 * rounding may change). DE_EINVAL if the shape does not fit. */
int de_set_launch(de_ctx *ctx, int32_t threads, int32_t vec4);
int de_get_launch(de_ctx *ctx, int32_t *threads, int32_t *vec4);

/* Base index rule: which rows form the mutant v = x_r0 + F (x_r1 - x_r2)
 * (Eq. 1; Section 2 lists several base index selections):
 *   DE_BASE_DISTINCT     r0, r1, r2 distinct and != i (DE/rand/1; default);
 *   DE_BASE_RANDOM       Alg. 3: r0 uniform over all rows (i included), then
 *                        Alg. 6: r1 = (r0 + k1) mod N, r2 = (r1 + k2) mod N with
 *                        k1, k2 uniform in [1, N - 1];
 *   DE_BASE_OFFSET       Alg. 4: r0 = (i + r_g) mod N, one r_g in [1, N - 1] per
 *                        generation, then Alg. 6;
 *   DE_BASE_PERMUTATION  Alg. 5: r0 = pi_g(i), a pseudorandom permutation of the
 *                        rows per generation (a keyed Feistel network with cycle
 *                        walking), then Alg. 6;
 *   DE_BASE_BEST         DE/best/1: r0 = the best row when the previous
 *                        generation closed (lowest value, lowest index), r1, r2
 *                        distinct and != i, != r0.
 * j_rand and the crossover draws do not depend on the rule. The debug draws
 * report (r0, r1, r2). Every rule draws from the row's IDX block; OFFSET and
 * PERMUTATION add a per-generation block (row field 2^32 - 1). */
typedef enum {
  DE_BASE_DISTINCT = 0,
  DE_BASE_RANDOM = 1,
  DE_BASE_OFFSET = 2,
  DE_BASE_PERMUTATION = 3,
  DE_BASE_BEST = 4
} de_base;

/* Set the base index rule of a context (every instance of a batch); it
 * applies from the next generation. DE_EINVAL for an unknown rule. */
int de_set_base(de_ctx *ctx, de_base base);
int de_get_base(de_ctx *ctx, de_base *base);

/* Generation kernel: 0 = automatic, 1 = one CTA per row (row held in
 * registers; every crossover, every D), 2 = persistent pipelined kernel (one
 * CTA per SM, a producer warp streams parent rows and the masked donor spans
 * into a shared-memory ring with bulk TMA copies; classic exponential and NEC
 * only; DE_EUNSUPPORTED for binomial or when a stage does not fit in shared
 * memory), 3 = streaming kernel (one warp per row, the row in chunks, the
 * trial recomputed and stored only when it wins; every crossover, every D).
 * Automatic picks 2 for exp / NEC and 3 for binomial when D >= 2048. Draws,
 * trials and selections are the same under every kernel; FP32 fitness
 * rounding differs by summation order. The rotated objectives ignore it. */
int de_set_kernel(de_ctx *ctx, int32_t kind);
/* The kernel in use: 1 or 2. */
int de_get_kernel(de_ctx *ctx, int32_t *kind);
/* Pipelined kernel shape: consumer threads per CTA (multiple of 32, 32..512;
 * default 256), shared-memory stages (2..8; 0 = as many as fit) and CTAs per
 * SM (1 or 2; two CTAs split the SM's shared memory; 0 = two when two stages
 * fit, else one). DE_EINVAL otherwise. */
int de_set_pipeline(de_ctx *ctx, int32_t consumer_threads, int32_t stages, int32_t ctas_per_sm);
/* The pipelined kernel's shape: consumer threads, stages, the floats of each
 * donor span buffer (segments longer than that read their donor genes from
 * global memory) and CTAs per SM; any pointer may be NULL. DE_EUNSUPPORTED
 * if the kernel is not available. */
int de_get_pipeline(de_ctx *ctx, int32_t *consumer_threads, int32_t *stages, int32_t *span_floats,
                    int32_t *ctas_per_sm);

/* ---- one generation without allocating ------------------------------------- */
/* The paper has no counterpart to this call; it serves callers that cannot
 * call cudaMalloc: plug-ins running inside another framework that owns every
 * device allocation and only lends buffers, code that must not implicitly
 * synchronise the device (cudaMalloc and cudaFree may), and programs that
 * reserve a fixed memory budget at start-up.
 *
 * One DE/rand/1/NEC generation on caller-owned device buffers; the call
 * allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 * Its scratch (generation state, slot bytes, NEC thresholds; 256 + 2*65536 +
 * 4*32768 bytes) is a fixed array compiled into the library, held by every GPU
 * that loads the library until the process exits.
 *   pop_in, pop_out: device, N rows of `pitch` floats (pitch >= D, a multiple
 *     of 4; both bases 16-byte aligned; distinct buffers); pop_in is read only.
 *   fit_in, fit_out: device, N floats (distinct buffers).
 *   Row i of pop_out / fit_out receives the trial and its FP32 fitness if the
 *   trial is strictly better than fit_in[i], else a copy of the parent row and
 *   fit_in[i]. Draws come from Philox with (seed, generation), as de_step's at
 *   that generation. For D < 2048 the call runs the kernel de_step runs, so
 *   pop_out and fit_out are bit-identical to what de_step computes from the
 *   same population; for D >= 2048 de_step's pipelined kernel sums the FP32
 *   fitness in another order, so fitness values may differ in the last bits
 *   (within 1e-5 max(1, |f|)) and a selection whose two values lie that
 *   close may differ; the trials themselves are identical.
 *   Objectives: sphere .. elliptic (Ackley constant 0.2); bounds as de_create.
 * Limits: 4 <= N <= 65536, 1 <= D <= 32768; larger sizes return DE_EINVAL.
 * Work is queued on `cuda_stream`. The first call on a device looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. Every call reuses
 * the same scratch and clears what must start at zero. The NEC thresholds are
 * rebuilt only when (Cr, D) differ from the previous call's on the device:
 * a chain of up to D - 1 dependent FP64 products, shorter the smaller Cr is
 * (measured on GB300: about 1.5 ms at D = 32768 with Cr = 0.9999, 0.03 ms
 * at Cr = 0.9), which only that call pays; a call with the thresholds kept
 * costs 0.03-0.05 ms at these sizes. Calls
 * that overlap on the GPU (different streams or host threads) race on the
 * scratch and must be serialised by the caller. */
int de_nec_step_noalloc(const float *pop_in, const float *fit_in, float *pop_out, float *fit_out,
                        int32_t N, int32_t D, int32_t pitch, float F, double CR, de_objective obj,
                        de_bounds b, uint64_t seed, int64_t generation, void *cuda_stream);

/* ---- crossover alone (Table I) --------------------------------------------- */
/* The crossover step by itself, as Table I times it, on caller-owned device
 * buffers; nothing is allocated and the work is queued on `cuda_stream`.
 * Row i (0 <= i < N) of generation `generation` gets the mask de_step uses for
 * row i at that generation with that seed and Philox instance field:
 *   bin: gene j crosses iff word j of the row's BIN stream < Cr 2^32, or
 *        j = j_rand (Eq. 2, Alg. 7);
 *   exp: the genes ((j - j_rand) mod D) < L, L from the sequential walk of
 *        Alg. 8 over the EXP stream;
 *   nec: the same circular segment with L from Eq. (9) (L = smallest n with
 *        Cr^n <= U, at most D; Alg. 9);
 * j_rand = word 3 of the row's IDX block scaled to [0, D). Each row's draws
 * depend only on (seed, generation, instance, i), not on N.
 * Arguments: 1 <= N, 1 <= D <= ld, 0 <= Cr <= 1, generation >= 0 (its low 32
 * bits enter the counter, as in de_step), instance < 2^24; DE_EINVAL
 * otherwise, DE_ECUDA if the launch fails. Errors of the queued work surface
 * at the caller's next synchronisation of the stream.
 *
 * de_crossover_mask: mask (device, N rows of ld bytes) gets 1 where gene j
 * crosses, 0 elsewhere; bytes j >= D of a row are not written.
 * de_crossover_apply: U = mask ? V : X elementwise (the trial matrix of Alg. 9 /
 * Alg. 10); u, x, v are device, N rows of ld floats; u must not alias x or v.
 * Elements j >= D of a row are neither read nor written. 16-byte aligned
 * bases with ld % 4 == 0 take 128-bit loads and stores. */
int de_crossover_mask(uint8_t *mask, int64_t ld, int32_t N, int32_t D, double CR, de_crossover xo,
                      uint64_t seed, int64_t generation, uint32_t instance, void *cuda_stream);
int de_crossover_apply(float *u, const float *x, const float *v, int64_t ld, int32_t N, int32_t D,
                       double CR, de_crossover xo, uint64_t seed, int64_t generation, uint32_t instance,
                       void *cuda_stream);

/* ---- misc ----------------------------------------------------------------- */
const char *de_strerror(int code);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int de_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DE_H */
