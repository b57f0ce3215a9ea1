/*
 * de_oracle.h — declarations of the plain CPU oracle for one DE/rand/1
 * generation (Pan, "Performance Analysis and Improvement of Parallel
 * Differential Evolution", arXiv 2101.06599).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path (the
 * CUDA library and its Python binding) never includes, links or calls it, and
 * this header shares nothing with the CUDA sources.
 *
 * All arrays are caller-owned, row-major, contiguous (row length D, no
 * padding). Functions never allocate memory that outlives the call.
 */
#ifndef DE_ORACLE_H
#define DE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Crossover kinds: binomial (Eq. 2 / Alg. 7), classic exponential (Alg. 8),
 * new exponential crossover NEC (Alg. 9 with Eq. 9). */
enum { OR_XO_BIN = 0, OR_XO_EXP = 1, OR_XO_NEC = 2 };

/* Objectives. 0-4 as printed in Section 4 (Ackley, Griewank, Rosenbrock) or
 * the textbook forms (sphere, Rastrigin); 5 = high-conditioned elliptic;
 * 6-7 = the shifted-rotated forms z = R (x - o). */
enum {
  OR_OBJ_SPHERE = 0, OR_OBJ_RASTRIGIN = 1, OR_OBJ_ACKLEY = 2,
  OR_OBJ_ROSENBROCK = 3, OR_OBJ_GRIEWANK = 4, OR_OBJ_ELLIPTIC = 5,
  OR_OBJ_SR_RASTRIGIN = 6, OR_OBJ_SR_ELLIPTIC = 7
};

/* Philox stream identifiers (top 8 bits of the fourth counter word). */
enum { OR_STREAM_INIT = 0, OR_STREAM_IDX = 1, OR_STREAM_LEN = 2,
       OR_STREAM_BIN = 3, OR_STREAM_EXP = 4, OR_STREAM_PERM = 5 };

/* Base index rules (Section 2 lists several; DE/rand/1 and DE/best/1):
 * DISTINCT     r1, r2, r3 distinct and != i (the default, DE/rand/1);
 * RANDOM       Alg. 3: r0 uniform over all rows, then Alg. 6: r1 = r0 + k1,
 *              r2 = r1 + k2 (mod N), k1, k2 uniform in [1, N-1];
 * OFFSET       Alg. 4: r0 = i + r_g (mod N), one r_g in [1, N-1] per
 *              generation, then Alg. 6;
 * PERMUTATION  Alg. 5: r0 = pi_g(i), a permutation of the rows per
 *              generation, then Alg. 6;
 * BEST         DE/best/1: r0 = the best row at the start of the generation,
 *              r1, r2 distinct, != i and != that row (the skip rule of the
 *              distinct donors with both excluded). */
enum { OR_BASE_DISTINCT = 0, OR_BASE_RANDOM = 1, OR_BASE_OFFSET = 2,
       OR_BASE_PERMUTATION = 3, OR_BASE_BEST = 4 };

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Word `idx` of stream `stream` for (seed, instance, generation g, row i):
 * word idx&3 of the block at counter (idx>>2, i, g, stream<<24 | inst). */
uint32_t or_word(uint64_t seed, uint32_t inst, uint32_t stream, int64_t g,
                 int32_t i, uint32_t idx);

/* Donors r[0..2] (distinct, all != i) and j_rand for row i. */
void or_donors(int32_t N, int32_t D, uint64_t seed, uint32_t inst, int64_t g,
               int32_t i, int32_t r[3], int32_t *jrand);

/* Base and difference indices of row i under a base rule (r[0] is the base
 * vector's row, r[1] and r[2] the difference rows) and j_rand. `best` is the
 * best row at the start of generation g (read by BEST only). */
void or_donors_base(int32_t N, int32_t D, uint64_t seed, uint32_t inst, int64_t g,
                    int32_t i, int base, int32_t best, int32_t r[3], int32_t *jrand);

/* Alg. 4's offset of generation g, in [1, N-1]. */
int32_t or_base_offset(int32_t N, uint64_t seed, uint32_t inst, int64_t g);

/* Alg. 5's permutation of generation g at row i. */
int32_t or_base_perm(int32_t N, uint64_t seed, uint32_t inst, int64_t g, int32_t i);

/* Eq. (9) for one uniform word w (U = w / 2^32). */
int32_t or_nec_length(uint32_t w, double Cr, int32_t D);

/* Alg. 8's continuation test on one word: 1 iff w / 2^32 < Cr. */
int or_exp_continues(uint32_t w, double Cr);

/* Alg. 8: number of genes the classic exponential crossover copies for row i. */
int32_t or_exp_length(uint64_t seed, uint32_t inst, int64_t g, int32_t i,
                      double Cr, int32_t D);

/* Crossover mask of row i (1 = gene taken from the mutant), and its L
 * (segment length for exp / NEC, number of set genes for bin). */
int32_t or_mask(int32_t D, double Cr, int xo, uint64_t seed, uint32_t inst,
                int64_t g, int32_t i, int32_t jrand, uint8_t *mask);

/* Objective value in FP64. `ackley_b` is the Ackley inner constant; `shift`
 * (D floats) and `rot` (D*D floats, row-major, z = R (x - o)) are only read
 * by the shifted-rotated objectives. */
double or_eval(int obj, int32_t D, const float *x, double ackley_b,
               const float *shift, const float *rot);

/* Uniform initial population in [lo, hi] from stream INIT. */
void or_init(int32_t N, int32_t D, float lo, float hi, uint64_t seed,
             uint32_t inst, float *pop);

/* One generation of Alg. 1 over rows [i0, i1) of an N x D population.
 * Rows outside the range are copied unchanged. Per-row outputs (may be NULL)
 * are indexed by i - i0: draws = 5 ints (r1, r2, r3, j_rand, L), trial =
 * D floats, ftrial = trial fitness, accept = 1 if the trial replaced the
 * parent, mask = D bytes. Returns 0, or -1 on invalid arguments. */
int or_step(int32_t N, int32_t D, float F, double Cr, int xo, int obj,
            float lo, float hi, uint64_t seed, uint32_t inst, int64_t g,
            double ackley_b, const float *shift, const float *rot,
            const float *pop_in, const double *fit_in,
            float *pop_out, double *fit_out, int32_t i0, int32_t i1,
            int32_t *draws, float *trial, double *ftrial, uint8_t *accept,
            uint8_t *mask);

/* or_step with a base index rule (`best` is read by OR_BASE_BEST only) and a
 * bound repair: 0 clips a mutant gene outside [lo, hi] to the violated
 * bound, 1 takes the midpoint between that bound and the target gene. */
int or_step_base(int32_t N, int32_t D, float F, double Cr, int xo, int obj,
                 float lo, float hi, uint64_t seed, uint32_t inst, int64_t g,
                 double ackley_b, const float *shift, const float *rot,
                 const float *pop_in, const double *fit_in,
                 float *pop_out, double *fit_out, int32_t i0, int32_t i1,
                 int32_t *draws, float *trial, double *ftrial, uint8_t *accept,
                 uint8_t *mask, int base, int32_t best, int repair);

/* Argmin of fit[0..N) with the lowest index winning ties; NaN counts as +inf. */
int32_t or_argmin(int32_t N, const double *fit);

#ifdef __cplusplus
}
#endif
#endif
