/*
 * de_oracle.c — plain, slow, obviously correct CPU oracle for one generation
 * of DE/rand/1 with binomial, classic exponential or new exponential (NEC)
 * crossover, after Pan, "Performance Analysis and Improvement of Parallel
 * Differential Evolution" (arXiv 2101.06599).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load or run this code. It shares no
 * source, header, table or helper with the CUDA library; both sides follow
 * the same written definitions (Philox4x32-10, the draw rules below, Eq. 1,
 * Eq. 2, Alg. 8, Eq. 9 with Alg. 9).
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off (no fast-math). With
 * contraction off and FLT_EVAL_METHOD 0 (x86-64 SSE, AArch64), every float
 * operation below rounds once to IEEE binary32, so the mutation is
 * fl(x_r1 + fl(F * fl(x_r2 - x_r3))) exactly.
 *
 * Structure: or_step follows Alg. 1 row by row — pick donors, mutate the
 * whole row (Eq. 1), repair bounds, recombine (Eq. 2, Alg. 8 or Alg. 9),
 * evaluate in FP64, keep the trial iff its fitness is strictly lower. The
 * paper states (Section 2, after Alg. 2) that this gives the same result as
 * the crossover-first parallel form the GPU uses.
 *
 * Readings where the paper is silent or garbled:
 *  - donors: r1, r2, r3 distinct and != i (replaces the index rules of
 *    Alg. 3 and Alg. 6, which as printed give constant indices);
 *  - random words: Philox4x32-10 with counter (block, i, g, stream<<24|inst)
 *    and key (seed lo, seed hi); rand(0,1) = w / 2^32 compared in FP64;
 *  - randint(m) = (w * m) >> 32 (multiply-shift, no rejection);
 *  - bound repair (the paper names none): clip to [lo, hi], or the midpoint
 *    between the violated bound and the target gene;
 *  - NaN fitness counts as +inf; ties keep the parent (strict '<', Alg. 1);
 *  - Alg. 10's mask formula as printed never wraps; the segment of Alg. 9
 *    (circular, starting at j_rand) is used instead.
 *  - Cr^n in Eq. (9) is evaluated as the FP64 product c_1 = Cr,
 *    c_n = fl(c_{n-1} * Cr).
 */
#include "de_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies with a     */
/* Weyl-sequence key schedule.                                               */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

uint32_t or_word(uint64_t seed, uint32_t inst, uint32_t stream, int64_t g,
                 int32_t i, uint32_t idx)
{
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = idx >> 2;
  ctr[1] = (uint32_t)i;
  ctr[2] = (uint32_t)g;
  ctr[3] = (stream << 24) | (inst & 0xFFFFFFu);
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  or_philox4x32_10(ctr, key, out);
  return out[idx & 3u];
}

/* rand(0,1) of the paper as an exact FP64 value w / 2^32 in [0, 1). */
static double unit_from_word(uint32_t w) { return (double)w / 4294967296.0; }

/* randint(m): an integer in [0, m) from one word. */
static int32_t randint_from_word(uint32_t w, int32_t m)
{
  return (int32_t)(((uint64_t)w * (uint64_t)(uint32_t)m) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Base / difference vector indices (DE/rand/1: u = x_r1 + F (x_r2 - x_r3),  */
/* Eq. 1) and j_rand (Alg. 7 and Alg. 10 both draw it).                     */
/* ------------------------------------------------------------------------ */
void or_donors(int32_t N, int32_t D, uint64_t seed, uint32_t inst, int64_t g,
               int32_t i, int32_t r[3], int32_t *jrand)
{
  uint32_t w[4];
  for (uint32_t k = 0; k < 4; k++) w[k] = or_word(seed, inst, OR_STREAM_IDX, g, i, k);

  /* excluded values, kept in ascending order */
  int32_t excl[4];
  int n_excl = 0;
  excl[n_excl++] = i;
  for (int k = 0; k < 3; k++) {
    /* the v-th value (0-based) of [0, N) with the excluded values removed */
    int32_t v = randint_from_word(w[k], N - 1 - k);
    for (int e = 0; e < n_excl; e++)
      if (v >= excl[e]) v++;
    r[k] = v;
    /* insert v keeping excl sorted */
    int pos = n_excl;
    while (pos > 0 && excl[pos - 1] > v) { excl[pos] = excl[pos - 1]; pos--; }
    excl[pos] = v;
    n_excl++;
  }
  *jrand = randint_from_word(w[3], D);
}

/* ------------------------------------------------------------------------ */
/* Base index rules. A per-generation draw uses the row field 2^32 - 1 of   */
/* the counter (no population row has that index).                         */
/* ------------------------------------------------------------------------ */
int32_t or_base_offset(int32_t N, uint64_t seed, uint32_t inst, int64_t g)
{
  uint32_t w = or_word(seed, inst, OR_STREAM_IDX, g, -1, 0);
  return 1 + randint_from_word(w, N - 1);
}

/* One Feistel round function on h-bit halves. */
static uint32_t feistel_f(uint32_t r, uint32_t k, uint32_t mask)
{
  uint32_t t = (r ^ k) * 0x9E3779B1u;
  t ^= t >> 15;
  t *= 0x2C1B3C6Du;
  t ^= t >> 13;
  return t & mask;
}

/* A bijection of [0, N): a 4-round Feistel network on 2h bits (the least
 * h >= 1 with 2^(2h) >= N), keyed by the 4 words of the generation's PERM
 * block, applied until the value falls in [0, N) (cycle walking: the orbit
 * of i under the bijection of [0, 2^(2h)) re-enters [0, N), and the first
 * element it meets there defines a bijection of [0, N)). */
int32_t or_base_perm(int32_t N, uint64_t seed, uint32_t inst, int64_t g, int32_t i)
{
  uint32_t k[4];
  for (uint32_t q = 0; q < 4; q++) k[q] = or_word(seed, inst, OR_STREAM_PERM, g, -1, q);
  int h = 1;
  while ((1ull << (2 * h)) < (uint64_t)N) h++;
  const uint32_t mask = (1u << h) - 1u;
  uint32_t x = (uint32_t)i;
  do {
    uint32_t L = x >> h, R = x & mask;
    for (int r = 0; r < 4; r++) {
      uint32_t nR = L ^ feistel_f(R, k[r], mask);
      L = R;
      R = nR;
    }
    x = (L << h) | R;
  } while (x >= (uint32_t)N);
  return (int32_t)x;
}

void or_donors_base(int32_t N, int32_t D, uint64_t seed, uint32_t inst, int64_t g,
                    int32_t i, int base, int32_t best, int32_t r[3], int32_t *jrand)
{
  if (base == OR_BASE_DISTINCT) {
    or_donors(N, D, seed, inst, g, i, r, jrand);
    return;
  }
  uint32_t w[4];
  for (uint32_t k = 0; k < 4; k++) w[k] = or_word(seed, inst, OR_STREAM_IDX, g, i, k);
  if (base == OR_BASE_BEST) {
    /* r1, r2: distinct, != i and != best, by the same skip rule as or_donors
       with {i, best} excluded from the start */
    int32_t excl[4];
    int n_excl = 0;
    excl[n_excl++] = i < best ? i : best;
    if (best != i) excl[n_excl++] = i < best ? best : i;
    r[0] = best;
    for (int k = 0; k < 2; k++) {
      int32_t v = randint_from_word(w[k], N - n_excl);
      for (int e = 0; e < n_excl; e++)
        if (v >= excl[e]) v++;
      r[1 + k] = v;
      int pos = n_excl;
      while (pos > 0 && excl[pos - 1] > v) { excl[pos] = excl[pos - 1]; pos--; }
      excl[pos] = v;
      n_excl++;
    }
    *jrand = randint_from_word(w[3], D);
    return;
  }
  int32_t r0;
  if (base == OR_BASE_RANDOM) r0 = randint_from_word(w[0], N);
  else if (base == OR_BASE_OFFSET) r0 = (int32_t)(((int64_t)i + or_base_offset(N, seed, inst, g)) % N);
  else r0 = or_base_perm(N, seed, inst, g, i);
  /* Alg. 6: each difference row a non-zero offset from the previous index */
  int32_t r1 = (int32_t)(((int64_t)r0 + 1 + randint_from_word(w[1], N - 1)) % N);
  int32_t r2 = (int32_t)(((int64_t)r1 + 1 + randint_from_word(w[2], N - 1)) % N);
  r[0] = r0; r[1] = r1; r[2] = r2;
  *jrand = randint_from_word(w[3], D);
}

/* ------------------------------------------------------------------------ */
/* Eq. (9): L = 1 if Cr = 0; D if Cr = 1; else min(ceil(ln U / ln Cr), D).   */
/* For U in (0,1) and Cr in (0,1), ceil(ln U / ln Cr) is the smallest n >= 1 */
/* with Cr^n <= U (multiplying n >= ln U / ln Cr by ln Cr < 0 flips it).     */
/* U = 0 gives ln U = -inf and therefore L = D; it is handled before the    */
/* loop because a long FP64 product Cr^n underflows to 0.                   */
/* ------------------------------------------------------------------------ */
int32_t or_nec_length(uint32_t w, double Cr, int32_t D)
{
  if (Cr <= 0.0) return 1;
  if (Cr >= 1.0) return D;
  double U = unit_from_word(w);
  if (U == 0.0) return D;        /* ln U = -inf: the ceiling is unbounded */
  int32_t n = 1;
  double crn = Cr;               /* Cr^n */
  while (n < D && !(crn <= U)) {
    n++;
    crn = crn * Cr;
  }
  return n;
}

/* Alg. 8's test after each copied gene: continue iff rand < Cr, with
 * rand = w / 2^32 compared with Cr in FP64 (both exact). */
int or_exp_continues(uint32_t w, double Cr)
{
  return unit_from_word(w) < Cr;
}

/* Alg. 8: copy one gene, then keep copying while rand < Cr and L < D. The
 * k-th draw (k = 1, 2, ...) is word k-1 of stream EXP for this row. Only the
 * number of copied genes is returned; the genes are j_rand, j_rand+1, ...
 * (mod D). */
int32_t or_exp_length(uint64_t seed, uint32_t inst, int64_t g, int32_t i,
                      double Cr, int32_t D)
{
  int32_t L = 0;
  uint32_t k = 0;
  int again;
  do {
    L = L + 1;                   /* u_j <- v_j ; j <- (j+1) mod D ; L++ */
    uint32_t w = or_word(seed, inst, OR_STREAM_EXP, g, i, k);
    k++;
    again = or_exp_continues(w, Cr) && (L < D);
  } while (again);
  return L;
}

int32_t or_mask(int32_t D, double Cr, int xo, uint64_t seed, uint32_t inst,
                int64_t g, int32_t i, int32_t jrand, uint8_t *mask)
{
  memset(mask, 0, (size_t)D);
  if (xo == OR_XO_BIN) {
    /* Eq. (2): gene j crosses if rand < Cr or j = j_rand; gene j uses word
     * j of stream BIN for this row. */
    int32_t cnt = 0;
    for (int32_t j = 0; j < D; j++) {
      double rnd = unit_from_word(or_word(seed, inst, OR_STREAM_BIN, g, i, (uint32_t)j));
      if (rnd < Cr || j == jrand) mask[j] = 1;
      cnt += mask[j];
    }
    return cnt;
  }
  int32_t L;
  if (xo == OR_XO_EXP) {
    L = or_exp_length(seed, inst, g, i, Cr, D);
  } else {
    uint32_t w = or_word(seed, inst, OR_STREAM_LEN, g, i, 0);
    L = or_nec_length(w, Cr, D);
  }
  /* Alg. 8 / Alg. 9: L consecutive genes from j_rand, wrapping at D. */
  int32_t j = jrand;
  int32_t l = 0;
  do {
    mask[j] = 1;
    j = (j + 1) % D;
    l = l + 1;
  } while (l < L);
  return L;
}

/* ------------------------------------------------------------------------ */
/* Objectives in FP64 (Section 4 for Ackley, Griewank and Rosenbrock).       */
/* ------------------------------------------------------------------------ */
static const double OR_PI = 3.14159265358979323846;
static const double OR_E = 2.71828182845904523536;

static double f_sphere(int32_t D, const double *x)
{
  double s = 0.0;
  for (int32_t j = 0; j < D; j++) s += x[j] * x[j];
  return s;
}

static double f_rastrigin(int32_t D, const double *x)
{
  double s = 10.0 * D;
  for (int32_t j = 0; j < D; j++) s += x[j] * x[j] - 10.0 * cos(2.0 * OR_PI * x[j]);
  return s;
}

static double f_ackley(int32_t D, const double *x, double b)
{
  double s2 = 0.0, sc = 0.0;
  for (int32_t j = 0; j < D; j++) {
    s2 += x[j] * x[j];
    sc += cos(2.0 * OR_PI * x[j]);
  }
  return -20.0 * exp(-b * sqrt(s2 / D)) - exp(sc / D) + 20.0 + OR_E;
}

static double f_rosenbrock(int32_t D, const double *x)
{
  double s = 0.0;
  for (int32_t j = 0; j + 1 < D; j++) {
    double a = x[j] * x[j] - x[j + 1];
    double c = 1.0 - x[j];
    s += 100.0 * a * a + c * c;
  }
  return s;
}

static double f_griewank(int32_t D, const double *x)
{
  double s = 0.0, p = 1.0;
  for (int32_t j = 0; j < D; j++) {
    s += x[j] * x[j] / 4000.0;
    p *= cos(x[j] / sqrt((double)(j + 1)));   /* j counted from 1 in the paper */
  }
  return s - p + 1.0;
}

static double f_elliptic(int32_t D, const double *x)
{
  double s = 0.0;
  for (int32_t j = 0; j < D; j++) {
    double c = (D > 1) ? pow(10.0, 6.0 * (double)j / (double)(D - 1)) : 1.0;
    s += c * x[j] * x[j];
  }
  return s;
}

double or_eval(int obj, int32_t D, const float *xf, double ackley_b,
               const float *shift, const float *rot)
{
  double *x = (double *)malloc((size_t)D * sizeof(double));
  if (!x) return NAN;
  if (obj == OR_OBJ_SR_RASTRIGIN || obj == OR_OBJ_SR_ELLIPTIC) {
    /* z = R (x - o), in FP64 from the FP32 inputs */
    for (int32_t k = 0; k < D; k++) {
      double z = 0.0;
      for (int32_t j = 0; j < D; j++)
        z += (double)rot[(size_t)k * D + j] * ((double)xf[j] - (double)shift[j]);
      x[k] = z;
    }
  } else {
    for (int32_t j = 0; j < D; j++) x[j] = (double)xf[j];
  }
  double f;
  switch (obj) {
    case OR_OBJ_SPHERE: f = f_sphere(D, x); break;
    case OR_OBJ_RASTRIGIN: case OR_OBJ_SR_RASTRIGIN: f = f_rastrigin(D, x); break;
    case OR_OBJ_ACKLEY: f = f_ackley(D, x, ackley_b); break;
    case OR_OBJ_ROSENBROCK: f = f_rosenbrock(D, x); break;
    case OR_OBJ_GRIEWANK: f = f_griewank(D, x); break;
    case OR_OBJ_ELLIPTIC: case OR_OBJ_SR_ELLIPTIC: f = f_elliptic(D, x); break;
    default: f = NAN; break;
  }
  free(x);
  return f;
}

/* ------------------------------------------------------------------------ */
/* Initial population (Alg. 1 / Alg. 2, first lines): uniform in [lo, hi]:   */
/* x = clip(lo + (hi - lo) * u), u = (w >> 8) * 2^-24, in FP32.              */
/* ------------------------------------------------------------------------ */
static float clip(float v, float lo, float hi)
{
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

void or_init(int32_t N, int32_t D, float lo, float hi, uint64_t seed,
             uint32_t inst, float *pop)
{
  float range = hi - lo;
  for (int32_t i = 0; i < N; i++)
    for (int32_t j = 0; j < D; j++) {
      uint32_t w = or_word(seed, inst, OR_STREAM_INIT, 0, i, (uint32_t)j);
      float u = (float)(w >> 8) * (1.0f / 16777216.0f);
      float t = range * u;
      float x = lo + t;
      pop[(size_t)i * D + j] = clip(x, lo, hi);
    }
}

/* Bound repair of a mutant gene v whose target gene is x (x in the box):
 * mode 0 clips to the violated bound; mode 1 takes the midpoint of that bound
 * and x, (bound + x) / 2 with each operation rounded once in FP32. */
static float repair_gene(float v, float x, float lo, float hi, int mode)
{
  if (v < lo) {
    if (!mode) return lo;
    float t = lo + x;
    return t * 0.5f;
  }
  if (v > hi) {
    if (!mode) return hi;
    float t = hi + x;
    return t * 0.5f;
  }
  return v;
}

static int fit_less(double a, double b)
{
  /* strict '<' with NaN read as +inf */
  if (isnan(a)) a = INFINITY;
  if (isnan(b)) b = INFINITY;
  return a < b;
}

int32_t or_argmin(int32_t N, const double *fit)
{
  int32_t best = 0;
  for (int32_t i = 1; i < N; i++)
    if (fit_less(fit[i], fit[best])) best = i;
  return best;
}

/* ------------------------------------------------------------------------ */
/* One generation, Alg. 1 row by row.                                       */
/* ------------------------------------------------------------------------ */
int or_step(int32_t N, int32_t D, float F, double Cr, int xo, int obj,
            float lo, float hi, uint64_t seed, uint32_t inst, int64_t g,
            double ackley_b, const float *shift, const float *rot,
            const float *pop_in, const double *fit_in,
            float *pop_out, double *fit_out, int32_t i0, int32_t i1,
            int32_t *draws, float *trial, double *ftrial, uint8_t *accept,
            uint8_t *mask_out)
{
  return or_step_base(N, D, F, Cr, xo, obj, lo, hi, seed, inst, g, ackley_b, shift, rot,
                      pop_in, fit_in, pop_out, fit_out, i0, i1, draws, trial, ftrial,
                      accept, mask_out, OR_BASE_DISTINCT, 0, 0);
}

int or_step_base(int32_t N, int32_t D, float F, double Cr, int xo, int obj,
                 float lo, float hi, uint64_t seed, uint32_t inst, int64_t g,
                 double ackley_b, const float *shift, const float *rot,
                 const float *pop_in, const double *fit_in,
                 float *pop_out, double *fit_out, int32_t i0, int32_t i1,
                 int32_t *draws, float *trial, double *ftrial, uint8_t *accept,
                 uint8_t *mask_out, int base, int32_t best, int repair)
{
  if (N < 4 || D < 1 || i0 < 0 || i1 > N || i0 > i1) return -1;
  if (repair != 0 && repair != 1) return -1;
  if (base < OR_BASE_DISTINCT || base > OR_BASE_BEST || best < 0 || best >= N) return -1;
  if (!(Cr >= 0.0 && Cr <= 1.0)) return -1;
  if (xo < OR_XO_BIN || xo > OR_XO_NEC) return -1;

  /* x_{g+1} starts as a copy of x_g; rows in [i0, i1) are then decided. */
  memcpy(pop_out, pop_in, (size_t)N * D * sizeof(float));
  memcpy(fit_out, fit_in, (size_t)N * sizeof(double));

  float *v = (float *)malloc((size_t)D * sizeof(float));
  float *u = (float *)malloc((size_t)D * sizeof(float));
  uint8_t *mask = (uint8_t *)malloc((size_t)D);
  if (!v || !u || !mask) { free(v); free(u); free(mask); return -1; }

  for (int32_t i = i0; i < i1; i++) {
    const float *xi = pop_in + (size_t)i * D;
    int32_t r[3], jrand;
    or_donors_base(N, D, seed, inst, g, i, base, best, r, &jrand);
    const float *x1 = pop_in + (size_t)r[0] * D;
    const float *x2 = pop_in + (size_t)r[1] * D;
    const float *x3 = pop_in + (size_t)r[2] * D;

    /* differential mutation, Eq. (1), every gene, then bound repair */
    for (int32_t j = 0; j < D; j++) {
      float diff = x2[j] - x3[j];
      float scaled = F * diff;
      float vj = x1[j] + scaled;
      v[j] = repair_gene(vj, xi[j], lo, hi, repair);
    }

    /* recombination: u starts as x_i; masked genes come from v */
    int32_t L = or_mask(D, Cr, xo, seed, inst, g, i, jrand, mask);
    for (int32_t j = 0; j < D; j++) u[j] = mask[j] ? v[j] : xi[j];

    double fu = or_eval(obj, D, u, ackley_b, shift, rot);
    int take = fit_less(fu, fit_in[i]);
    if (take) {
      memcpy(pop_out + (size_t)i * D, u, (size_t)D * sizeof(float));
      fit_out[i] = fu;
    }

    int32_t k = i - i0;
    if (draws) {
      draws[5 * k + 0] = r[0];
      draws[5 * k + 1] = r[1];
      draws[5 * k + 2] = r[2];
      draws[5 * k + 3] = jrand;
      draws[5 * k + 4] = L;
    }
    if (trial) memcpy(trial + (size_t)k * D, u, (size_t)D * sizeof(float));
    if (ftrial) ftrial[k] = fu;
    if (accept) accept[k] = (uint8_t)take;
    if (mask_out) memcpy(mask_out + (size_t)k * D, mask, (size_t)D);
  }
  free(v);
  free(u);
  free(mask);
  return 0;
}
