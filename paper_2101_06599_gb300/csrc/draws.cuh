// draws.cuh — integer-exact draw rules of one generation (device side).
//
// All randomness is Philox words; every rule below is integer arithmetic,
// so any two implementations of the same rules agree bit for bit.
//
//  - randint(m) = (w * m) >> 32 (multiply-shift; bias <= m / 2^32).
//  - Donors (DE/rand/1, Eq. 1): r1 = randint(N-1) on word 0 of the row's IDX
//    block, then every excluded value e <= r1 in ascending order shifts it up
//    by one (excluded = {i}); r2 likewise from word 1 with {i, r1}, r3 from
//    word 2 with {i, r1, r2}: uniform over ordered distinct triples, != i.
//  - j_rand = randint(D) on word 3 (Alg. 7 and Alg. 10 both draw it).
//  - rand(0,1) < Cr is w < ceil(Cr * 2^32), i.e. w / 2^32 < Cr exactly.
//  - NEC length, Eq. (9): for U = w / 2^32 in (0, 1) and Cr in (0, 1),
//    ceil(ln U / ln Cr) = 1 + #{n >= 1 : U < Cr^n}. With Cr^n taken as the
//    FP64 product c_n = fl(c_{n-1} Cr) and T_n = ceil(c_n 2^32),
//    U < c_n  <=>  w < T_n  <=>  w <= T_n - 1, and T_n does not increase
//    with n, so L = 1 + n*, n* = the largest n <= D - 1 with w <= T_n - 1
//    (0 if none), read from a table of T_n - 1. The table stops before the
//    first T_n <= 1 (no w >= 1 passes it); w = 0 is U = 0, where ln U = -inf
//    and L = D. Cr = 0 gives L = 1 and Cr = 1 gives L = D.
//    The lookup is O(1): the real-valued form of the same count, n* =
//    ceil(x) - 1 with x = log2(U) / log2(Cr) = (32 - log2 w) / (-log2 Cr),
//    gives a first guess, and the table entries on either side of the guess
//    confirm it (one pair of loads) or move it to the exact count. The
//    result is the table's, whatever the guess, so it stays bit-exact.
//  - Classic exponential crossover (Alg. 8): after copying L genes the walk
//    draws word L-1 of the row's EXP stream and continues iff w < ceil(Cr
//    2^32) and L < D.
#pragma once
#include "common.cuh"

namespace de {

__device__ __forceinline__ int randint_w(uint32_t w, uint32_t m) {
  return (int)(((unsigned long long)w * (unsigned long long)m) >> 32);
}

struct RowDraws {
  int r1, r2, r3, jrand, L;
};

// One Feistel round on h-bit halves (the permutation base rule).
__device__ __forceinline__ uint32_t feistel_f(uint32_t r, uint32_t k, uint32_t mask) {
  uint32_t t = (r ^ k) * 0x9E3779B1u;
  t ^= t >> 15;
  t *= 0x2C1B3C6Du;
  t ^= t >> 13;
  return t & mask;
}

// Alg. 5's permutation of generation g at row i: a 4-round Feistel network on
// 2h bits (the least h >= 1 with 2^(2h) >= N) keyed by the generation's PERM
// block, applied until the value falls in [0, N) (cycle walking; at most
// 2^(2h) - N steps, fewer than 3N).
__device__ __forceinline__ int base_permutation(const GenParams& p, uint32_t g, int i) {
  const uint4 k = philox_block(p.key, kStreamPerm, p.inst, g, 0xFFFFFFFFu, 0u);
  int h = 1;
  while ((1ull << (2 * h)) < (unsigned long long)p.N) ++h;
  const uint32_t mask = (1u << h) - 1u;
  uint32_t x = (uint32_t)i;
  do {
    uint32_t L = x >> h, R = x & mask;
    uint32_t nR = L ^ feistel_f(R, k.x, mask); L = R; R = nR;
    nR = L ^ feistel_f(R, k.y, mask); L = R; R = nR;
    nR = L ^ feistel_f(R, k.z, mask); L = R; R = nR;
    nR = L ^ feistel_f(R, k.w, mask); L = R; R = nR;
    x = (L << h) | R;
  } while (x >= (uint32_t)p.N);
  return (int)x;
}

// Rows of row i under the base rules other than the default (Section 2's
// base index selections, Alg. 3-5, with Alg. 6's difference indices; and
// DE/best/1): d.r1 is the base vector's row, d.r2 and d.r3 the difference
// rows. Every rule takes j_rand from word 3 of the row's IDX block.
static __device__ __noinline__ void draw_donors_rule(const GenParams& p, uint32_t g, int i, const uint4 b, RowDraws& d) {
  if (p.base == kBaseBest) {
    int best = p.st->base_row;
    if (best < 0 || best >= p.N) best = 0;
    // two draws by the skip rule with {i, best} excluded from the start
    int e0 = min(i, best), e1 = max(i, best);
    const int nex = (best != i) ? 2 : 1;
    int v = randint_w(b.x, (uint32_t)(p.N - nex));
    v += (v >= e0);
    if (nex == 2) v += (v >= e1);
    const int r2 = v;
    int f0, f1, f2;                                // sorted {e0, (e1), r2}
    if (nex == 2) {
      if (r2 < e0) { f0 = r2; f1 = e0; f2 = e1; }
      else if (r2 < e1) { f0 = e0; f1 = r2; f2 = e1; }
      else { f0 = e0; f1 = e1; f2 = r2; }
    } else {
      f0 = min(e0, r2); f1 = max(e0, r2); f2 = 0x7FFFFFFF;
    }
    v = randint_w(b.y, (uint32_t)(p.N - nex - 1));
    v += (v >= f0);
    v += (v >= f1);
    if (nex == 2) v += (v >= f2);
    d.r1 = best;
    d.r2 = r2;
    d.r3 = v;
  } else {
    int r0;
    if (p.base == kBaseRandom) {
      r0 = randint_w(b.x, (uint32_t)p.N);
    } else if (p.base == kBaseOffset) {
      const uint32_t w = philox_block(p.key, kStreamIdx, p.inst, g, 0xFFFFFFFFu, 0u).x;
      r0 = (int)(((long long)i + 1 + randint_w(w, (uint32_t)(p.N - 1))) % p.N);
    } else {
      r0 = base_permutation(p, g, i);
    }
    const int r1 = (int)(((long long)r0 + 1 + randint_w(b.y, (uint32_t)(p.N - 1))) % p.N);
    const int r2 = (int)(((long long)r1 + 1 + randint_w(b.z, (uint32_t)(p.N - 1))) % p.N);
    d.r1 = r0;
    d.r2 = r1;
    d.r3 = r2;
  }
  d.jrand = randint_w(b.w, (uint32_t)p.D);
}

// Donors and j_rand of row i in generation g.
__device__ __forceinline__ void draw_donors(const GenParams& p, uint32_t g, int i, RowDraws& d) {
  const uint4 b = philox_block(p.key, kStreamIdx, p.inst, g, (uint32_t)i, 0u);
  if (p.base != kBaseDistinct) {
    draw_donors_rule(p, g, i, b, d);
    return;
  }
  int e0 = i;                                  // sorted excluded values e0 < e1 < e2
  int v = randint_w(b.x, (uint32_t)(p.N - 1));
  v += (v >= e0);
  d.r1 = v;
  int e1;
  if (v < e0) { e1 = e0; e0 = v; } else { e1 = v; }
  v = randint_w(b.y, (uint32_t)(p.N - 2));
  v += (v >= e0);
  v += (v >= e1);
  d.r2 = v;
  int e2;
  if (v < e0) { e2 = e1; e1 = e0; e0 = v; }
  else if (v < e1) { e2 = e1; e1 = v; }
  else { e2 = v; }
  v = randint_w(b.z, (uint32_t)(p.N - 3));
  v += (v >= e0);
  v += (v >= e1);
  v += (v >= e2);
  d.r3 = v;
  d.jrand = randint_w(b.w, (uint32_t)p.D);
}

// Eq. (9) from the LEN word w of a row: L = 1 + n*, n* = #{1 <= n <= nmax :
// w <= tm1[n - 1]} (a prefix of n, the table being non-increasing), with
// nmax = min(D - 1, nT) and kinv = 1 / -log2(Cr). kShared: tm1 is in shared
// memory (else global, read through the read-only path).
template <bool kShared>
__device__ __forceinline__ uint32_t nec_tab_at(const uint32_t* tm1, int k) {
  if constexpr (kShared) return tm1[k];
  else return __ldg(tm1 + k);
}

template <bool kShared>
__device__ __forceinline__ int nec_length_word(uint32_t w, const uint32_t* tm1, int nmax, int D, float kinv) {
  if (w == 0u) return D;                                   // U = 0: ln U = -inf
  const float x = (32.0f - __log2f((float)w)) * kinv;     // log2(U) / log2(Cr)
  int n = (int)ceilf(x) - 1;                               // the guess of n*
  n = max(0, min(n, nmax));
  // n* = n iff n passes (n = 0 always does) and n + 1 does not (or n = nmax)
  const uint32_t below = (n > 0) ? nec_tab_at<kShared>(tm1, n - 1) : 0xFFFFFFFFu;
  const uint32_t above = (n < nmax) ? nec_tab_at<kShared>(tm1, n) : 0u;
  if (w <= below && w > above) return 1 + n;
  while (n < nmax && w <= nec_tab_at<kShared>(tm1, n)) ++n;        // guess too low
  while (n > 0 && w > nec_tab_at<kShared>(tm1, n - 1)) --n;        // guess too high
  return 1 + n;
}

// L of row i in generation g from its Cr mode and a given LEN word.
template <bool kShared>
__device__ __forceinline__ int nec_length_of(const GenParams& p, uint32_t w, const uint32_t* tm1) {
  if (p.cr_mode == kCrZero) return 1;
  if (p.cr_mode == kCrOne) return p.D;
  return nec_length_word<kShared>(w, tm1, min(p.D - 1, p.nT), p.D, p.nec_k);
}

__device__ __forceinline__ uint32_t nec_word(const GenParams& p, uint32_t g, int i) {
  return philox_block(p.key, kStreamLen, p.inst, g, (uint32_t)i, 0u).x;
}

// NEC segment length of row i, Eq. (9), through the table in global memory.
__device__ __forceinline__ int nec_length(const GenParams& p, uint32_t g, int i) {
  if (p.cr_mode != kCrGeneral) return p.cr_mode == kCrZero ? 1 : p.D;
  return nec_length_of<false>(p, nec_word(p, g, i), p.nec_tm1);
}

// Binomial mask bits of slot q (genes 4q .. 4q+3, bit e = gene 4q + e) from
// the slot's BIN block w (Eq. 2): word e < ceil(Cr 2^32), and the gene j_rand
// always. Padding genes are the caller's to clear.
__device__ __forceinline__ unsigned bin_mask(const GenParams& p, const uint4 w, int q, int jrand) {
  unsigned m = (w.x < p.cr_lt ? 1u : 0u) | (w.y < p.cr_lt ? 2u : 0u) | (w.z < p.cr_lt ? 4u : 0u) |
               (w.w < p.cr_lt ? 8u : 0u);
  if (p.cr_all) m = 0xFu;
  if (q == (jrand >> 2)) m |= 1u << (jrand & 3);
  return m;
}

// Alg. 8's continuation test for one EXP word: rand < Cr, i.e. w < ceil(Cr 2^32).
__device__ __forceinline__ bool exp_continues(const GenParams& p, uint32_t w) {
  return (unsigned long long)w < p.cr_t;
}

// Alg. 8's sequential walk: returns L.
__device__ __forceinline__ int exp_walk_length(const GenParams& p, uint32_t g, int i) {
  int L = 1;
  uint32_t k = 0;
  uint4 blk = make_uint4(0, 0, 0, 0);
  while (L < p.D) {
    if ((k & 3u) == 0u) blk = philox_block(p.key, kStreamExp, p.inst, g, (uint32_t)i, k >> 2);
    const uint32_t w = word_of(blk, k & 3u);
    ++k;
    if (!exp_continues(p, w)) break;
    ++L;
  }
  return L;
}

}  // namespace de
