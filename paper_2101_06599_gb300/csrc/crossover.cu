// crossover.cu — crossover alone, the operation Table I times: for every row
// i of an N x D matrix, the mask of binomial crossover (Eq. 2), classic
// exponential crossover (Alg. 8) or the new exponential crossover (Eq. 9 with
// the circular segment of Alg. 9), either materialised as bytes or applied to
// a target matrix X and a mutant matrix V (U = mask ? V : X). The draws are
// the ones de_step uses at the same (seed, generation, instance): j_rand is
// word 3 of the row's IDX block, L comes from the LEN stream (NEC) or the
// sequential walk over the EXP stream (exp), binomial gene j uses word j of
// the BIN stream.
//
// One warp per row, 8 rows per CTA: lane 0 draws j_rand and L, the lanes
// cover the row 4 genes at a time. NEC's L is computed here without the
// threshold table: L = 1 + #{n >= 1 : w < c_n 2^32} with c_1 = Cr and
// c_n = fl(c_{n-1} Cr) in FP64 (a plain IEEE multiply, the same numbers the
// table holds), counted until the first n that fails (c_n decreases).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/de.h"
#include "draws.cuh"
#include "internal.h"

namespace de {

constexpr int kXoWarps = 8;

__device__ __forceinline__ int nec_length_fp64(const GenParams& p, double cr, uint32_t g, int i) {
  if (p.cr_mode == kCrZero) return 1;
  if (p.cr_mode == kCrOne) return p.D;
  const uint32_t w = philox_block(p.key, kStreamLen, p.inst, g, (uint32_t)i, 0u).x;
  if (w == 0u) return p.D;                          // U = 0: ln U = -inf
  const double wd = (double)w;
  int L = 1;
  double c = cr;
  while (L < p.D && wd < c * 4294967296.0) {
    ++L;
    c = c * cr;
  }
  return L;
}

// j_rand and L of row i (lane 0 computes, every lane receives them).
template <int XO>
__device__ __forceinline__ void xo_row_draws(const GenParams& p, double cr, uint32_t g, int i, int lane,
                                             int& jrand, int& L) {
  int j = 0, l = 0;
  if (lane == 0) {
    const uint4 b = philox_block(p.key, kStreamIdx, p.inst, g, (uint32_t)i, 0u);
    j = randint_w(b.w, (uint32_t)p.D);
    if constexpr (XO == kNec) l = nec_length_fp64(p, cr, g, i);
    else if constexpr (XO == kExp) l = exp_walk_length(p, g, i);
  }
  jrand = __shfl_sync(0xFFFFFFFFu, j, 0);
  L = __shfl_sync(0xFFFFFFFFu, l, 0);
}

// Mask bits of genes 4q .. 4q+3 of row i (bit e = gene 4q + e; genes >= D clear).
template <int XO>
__device__ __forceinline__ unsigned xo_slot_mask(const GenParams& p, uint32_t g, int i, int q, int jrand, int L) {
  const int j0 = 4 * q;
  unsigned m = 0u;
  if constexpr (XO == kBin) {
    const uint4 w = philox_block(p.key, kStreamBin, p.inst, g, (uint32_t)i, (uint32_t)q);
    m |= ((unsigned long long)w.x < p.cr_t || j0 + 0 == jrand) ? 1u : 0u;
    m |= ((unsigned long long)w.y < p.cr_t || j0 + 1 == jrand) ? 2u : 0u;
    m |= ((unsigned long long)w.z < p.cr_t || j0 + 2 == jrand) ? 4u : 0u;
    m |= ((unsigned long long)w.w < p.cr_t || j0 + 3 == jrand) ? 8u : 0u;
  } else {
    int dd = j0 - jrand;
    if (dd < 0) dd += p.D;                          // (j0 - j_rand) mod D
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int de = dd + e;
      if (de >= p.D) de -= p.D;
      m |= (de < L) ? (1u << e) : 0u;
    }
  }
  return m & ((1u << min(4, p.D - j0)) - 1u);
}

// VEC: ld % 4 == 0 and the base 4-byte aligned (one 4-byte store per slot).
template <int XO, bool VEC>
__global__ void __launch_bounds__(kXoWarps * 32) xo_mask_kernel(const __grid_constant__ GenParams p, double cr,
                                                                uint32_t g, uint8_t* __restrict__ mask,
                                                                long long ld) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kXoWarps + (threadIdx.x >> 5);
  if (i >= p.N) return;                             // warp-uniform
  int jrand, L;
  xo_row_draws<XO>(p, cr, g, i, lane, jrand, L);
  uint8_t* row = mask + (size_t)i * (size_t)ld;
  for (int q = lane; q < p.D4; q += 32) {
    const unsigned m = xo_slot_mask<XO>(p, g, i, q, jrand, L);
    const unsigned bytes = (m & 1u) | ((m & 2u) << 7) | ((m & 4u) << 14) | ((m & 8u) << 21);
    if (VEC && 4 * q + 4 <= p.D) {
      *reinterpret_cast<uint32_t*>(row + 4 * q) = bytes;
    } else {
      for (int e = 0; e < 4 && 4 * q + e < p.D; ++e) row[4 * q + e] = (uint8_t)((m >> e) & 1u);
    }
  }
}

// VEC: ld % 4 == 0 and all three bases 16-byte aligned (float4 loads and stores).
template <int XO, bool VEC>
__global__ void __launch_bounds__(kXoWarps * 32) xo_apply_kernel(const __grid_constant__ GenParams p, double cr,
                                                                 uint32_t g, float* __restrict__ u,
                                                                 const float* __restrict__ x,
                                                                 const float* __restrict__ v, long long ld) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kXoWarps + (threadIdx.x >> 5);
  if (i >= p.N) return;                             // warp-uniform
  int jrand, L;
  xo_row_draws<XO>(p, cr, g, i, lane, jrand, L);
  const size_t base = (size_t)i * (size_t)ld;
  const int full4 = VEC ? p.D / 4 : 0;              // slots whose 4 genes are all < D
  constexpr int U = 4;                               // slots per lane in flight
  int q0 = 0;
  for (; q0 + 32 * U <= full4; q0 += 32 * U) {
    float4 xv[U], vv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int j0 = 4 * (q0 + lane + 32 * k);
      xv[k] = ld_stream(reinterpret_cast<const float4*>(x + base + j0));
      vv[k] = ld_stream(reinterpret_cast<const float4*>(v + base + j0));
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int q = q0 + lane + 32 * k;
      const unsigned m = xo_slot_mask<XO>(p, g, i, q, jrand, L);
      float4 o;
      o.x = (m & 1u) ? vv[k].x : xv[k].x;
      o.y = (m & 2u) ? vv[k].y : xv[k].y;
      o.z = (m & 4u) ? vv[k].z : xv[k].z;
      o.w = (m & 8u) ? vv[k].w : xv[k].w;
      st_stream(reinterpret_cast<float4*>(u + base + 4 * q), o);
    }
  }
  for (int q = q0 + lane; q < p.D4; q += 32) {
    const unsigned m = xo_slot_mask<XO>(p, g, i, q, jrand, L);
    const int j0 = 4 * q;
    if (VEC && j0 + 4 <= p.D) {
      const float4 xv = ld_stream(reinterpret_cast<const float4*>(x + base + j0));
      const float4 vv = ld_stream(reinterpret_cast<const float4*>(v + base + j0));
      float4 o;
      o.x = (m & 1u) ? vv.x : xv.x;
      o.y = (m & 2u) ? vv.y : xv.y;
      o.z = (m & 4u) ? vv.z : xv.z;
      o.w = (m & 8u) ? vv.w : xv.w;
      st_stream(reinterpret_cast<float4*>(u + base + j0), o);
    } else {
      for (int e = 0; e < 4 && j0 + e < p.D; ++e)
        u[base + j0 + e] = ((m >> e) & 1u) ? v[base + j0 + e] : x[base + j0 + e];
    }
  }
}

}  // namespace de

using namespace de;

namespace {

bool xo_args_ok(int64_t ld, int32_t N, int32_t D, double CR, int xo, int64_t generation, uint32_t instance) {
  if (N < 1 || D < 1 || ld < D) return false;
  if (!(CR >= 0.0 && CR <= 1.0)) return false;
  if (xo != DE_XOVER_BIN && xo != DE_XOVER_EXP && xo != DE_XOVER_NEC) return false;
  if (generation < 0 || instance >= (1u << 24)) return false;
  return true;
}

GenParams xo_params(int32_t N, int32_t D, double CR, uint64_t seed, uint32_t instance) {
  GenParams p;
  std::memset(&p, 0, sizeof(p));
  p.N = N;
  p.D = D;
  p.D4 = (D + 3) / 4;
  p.cr_mode = (CR <= 0.0) ? kCrZero : (CR >= 1.0 ? kCrOne : kCrGeneral);
  p.cr_t = (unsigned long long)std::ceil(CR * 4294967296.0);
  p.cr_lt = (uint32_t)std::min<unsigned long long>(p.cr_t, 0xFFFFFFFFull);
  p.cr_all = p.cr_t > 0xFFFFFFFFull ? 1 : 0;
  p.key = Key2{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
  p.rk = philox_round_keys(p.key);
  p.inst = instance;
  return p;
}

template <bool VEC>
cudaError_t launch_mask(int xo, const GenParams& p, double cr, uint32_t g, uint8_t* mask, long long ld,
                        cudaStream_t s) {
  const unsigned grid = (unsigned)((p.N + kXoWarps - 1) / kXoWarps);
  if (xo == DE_XOVER_BIN) xo_mask_kernel<kBin, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, mask, ld);
  else if (xo == DE_XOVER_EXP) xo_mask_kernel<kExp, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, mask, ld);
  else xo_mask_kernel<kNec, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, mask, ld);
  return cudaGetLastError();
}

template <bool VEC>
cudaError_t launch_apply(int xo, const GenParams& p, double cr, uint32_t g, float* u, const float* x,
                         const float* v, long long ld, cudaStream_t s) {
  const unsigned grid = (unsigned)((p.N + kXoWarps - 1) / kXoWarps);
  if (xo == DE_XOVER_BIN) xo_apply_kernel<kBin, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, u, x, v, ld);
  else if (xo == DE_XOVER_EXP) xo_apply_kernel<kExp, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, u, x, v, ld);
  else xo_apply_kernel<kNec, VEC><<<grid, kXoWarps * 32, 0, s>>>(p, cr, g, u, x, v, ld);
  return cudaGetLastError();
}

}  // namespace

extern "C" int de_crossover_mask(uint8_t* mask, int64_t ld, int32_t N, int32_t D, double CR, de_crossover xo,
                                 uint64_t seed, int64_t generation, uint32_t instance, void* cuda_stream) {
  if (!mask || !xo_args_ok(ld, N, D, CR, (int)xo, generation, instance)) return DE_EINVAL;
  const GenParams p = xo_params(N, D, CR, seed, instance);
  const uint32_t g = (uint32_t)generation;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(mask) & 3u) == 0);
  const cudaError_t e = vec ? launch_mask<true>((int)xo, p, CR, g, mask, ld, s)
                            : launch_mask<false>((int)xo, p, CR, g, mask, ld, s);
  return e == cudaSuccess ? DE_OK : DE_ECUDA;
}

extern "C" int de_crossover_apply(float* u, const float* x, const float* v, int64_t ld, int32_t N, int32_t D, double CR,
                            de_crossover xo, uint64_t seed, int64_t generation, uint32_t instance,
                            void* cuda_stream) {
  if (!u || !x || !v || !xo_args_ok(ld, N, D, CR, (int)xo, generation, instance)) return DE_EINVAL;
  if (u == x || u == v) return DE_EINVAL;
  const GenParams p = xo_params(N, D, CR, seed, instance);
  const uint32_t g = (uint32_t)generation;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const uintptr_t a = reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(x) |
                      reinterpret_cast<uintptr_t>(v);
  const bool vec = (ld % 4 == 0) && ((a & 15u) == 0);
  const cudaError_t e = vec ? launch_apply<true>((int)xo, p, CR, g, u, x, v, ld, s)
                            : launch_apply<false>((int)xo, p, CR, g, u, x, v, ld, s);
  return e == cudaSuccess ? DE_OK : DE_ECUDA;
}
