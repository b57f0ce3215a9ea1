// philox.cuh — Philox4x32-10 counter-based generator for the device.
//
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds; each round multiplies counter words 0 and 2 by two
// fixed 32-bit constants, XORs the high halves with the other two words and
// the round key, and the key advances by a Weyl increment per round.
//
// Counter layout used by the library: (block, row, generation, stream<<24 |
// instance), key = (seed low word, seed high word). A draw is a pure
// function of those values, which is what makes results independent of the
// launch shape and lets checkpoints resume bit-identically.
#pragma once
#include <cstdint>

namespace de {

enum : uint32_t {
  kStreamInit = 0u,  // initial population
  kStreamIdx = 1u,   // r1, r2, r3, j_rand (one block per row)
  kStreamLen = 2u,   // NEC segment length (word 0)
  kStreamBin = 3u,   // binomial crossover: word j for gene j
  kStreamExp = 4u,   // classic exponential crossover: word k for step k+1
  kStreamPerm = 5u,  // permutation base rule: Feistel keys of a generation
};

struct Key2 { uint32_t k0, k1; };

// The key schedule: round r (r = 0 .. 9) uses (k0 + r A, k1 + r B) mod 2^32,
// A, B the Weyl increments. Precomputed once per context, it saves the
// per-round key additions of kernels that draw one block per few genes.
constexpr uint32_t kPhiloxBumpA = 0x9E3779B9u, kPhiloxBumpB = 0xBB67AE85u;
struct RoundKeys { uint32_t k[20]; };

__host__ __device__ inline RoundKeys philox_round_keys(Key2 key) {
  RoundKeys rk;
  uint32_t k0 = key.k0, k1 = key.k1;
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += kPhiloxBumpA;
    k1 += kPhiloxBumpB;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, Key2 key) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  constexpr uint32_t kBumpA = kPhiloxBumpA, kBumpB = kPhiloxBumpB;
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
    const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
    c = make_uint4(hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA);
    k0 += kBumpA;
    k1 += kBumpB;
  }
  return c;
}

// The same ten rounds with the round keys read from a precomputed schedule.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys& rk) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
    const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
    c = make_uint4(hiB ^ c.y ^ rk.k[2 * r], loB, hiA ^ c.w ^ rk.k[2 * r + 1], loA);
  }
  return c;
}

// The block of stream `stream` at counter word 0 = `block` for row `row` in
// generation `gen` of instance `inst`.
__device__ __forceinline__ uint4 philox_block(Key2 key, uint32_t stream, uint32_t inst,
                                              uint32_t gen, uint32_t row, uint32_t block) {
  return philox4x32_10(make_uint4(block, row, gen, (stream << 24) | (inst & 0xFFFFFFu)), key);
}

__device__ __forceinline__ uint32_t word_of(const uint4& b, uint32_t w) {
  return w == 0 ? b.x : (w == 1 ? b.y : (w == 2 ? b.z : b.w));
}

__device__ __forceinline__ uint4 philox_block_rk(const RoundKeys& rk, uint32_t stream, uint32_t inst,
                                                 uint32_t gen, uint32_t row, uint32_t block) {
  return philox4x32_10_rk(make_uint4(block, row, gen, (stream << 24) | (inst & 0xFFFFFFu)), rk);
}

}  // namespace de
