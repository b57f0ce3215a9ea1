// sr_kernels.cu — generation of the shifted-rotated objectives.
//
// One generation = sr_trial_kernel (draws, crossover, mutation, clipping as
// in the separable path; the trial row is written to the row's other slot
// buffer, so acceptance is a slot flip; a = u - o and |a|^2, and for the BF16
// path the split operands bf16(a), bf16(a - bf16(a))), then the product
// Z = A R^T with a fused g(z) epilogue (this file: FP32 SIMT; sr_tc.cu:
// tcgen05), then sr_select_kernel (strict '<' decisions, or interval
// decisions with a per-row error bound on the BF16 path: rows whose interval
// straddles the parent's go to an FP32 re-evaluation with this file's GEMM
// and sr_resolve_kernel), then sr_finish_kernel (FP64 incumbent when due, and
// the close of the generation).
//
// The FP32 GEMM accumulates every z_ik in one fixed order (j ascending, one
// FMA per term, one thread per element) and reduces g(z) over each 64-column
// tile in one fixed order, so a row's value does not depend on which other
// rows share its tile: re-evaluating a row reproduces the FP32 path bit for
// bit.
#include "draws.cuh"
#include "gen_kernel.cuh"
#include "internal.h"
#include "sr_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace de {

// ---------------------------------------------------------------------------
// trials: one warp per row, 8 rows per CTA. The warp issues its first parent
// loads, lane 0 draws the donors and L (Philox, slot lookups) and broadcasts
// them, then the lanes stream the row 4 genes at a time: crossover mask,
// mutation and clip of masked genes, the trial into the other slot, a = u - o
// with |a|^2, and on the BF16 path the split operands as packed 8-byte
// stores. Mask counts go to the state with one atomic per CTA.
// ---------------------------------------------------------------------------
constexpr int kTrialWarps = 8, kTrialUnroll = 4;

template <int XO>
__global__ void __launch_bounds__(kTrialWarps * 32, 4) sr_trial_kernel(const __grid_constant__ SrParams sp) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  __shared__ int wcnt[kTrialWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kTrialWarps + warp;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  int Lrow = 0;
  if (i < p.N) {                                   // warp-uniform
    const int si = slot_in[i];
    const float4* xrow = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)i * p.pitch);
    float4* trow = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
    float4 x[kTrialUnroll];
#pragma unroll
    for (int u = 0; u < kTrialUnroll; ++u) {
      const int q = lane + 32 * u;
      x[u] = (q < p.D4) ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    RowDraws d{};
    unsigned long long pd1 = 0, pd2 = 0, pd3 = 0;
    if (lane == 0) {
      draw_donors(p, g, i, d);
      if constexpr (XO == kNec) d.L = nec_length(p, g, i);
      else if constexpr (XO == kExp) d.L = exp_walk_length(p, g, i);
      else d.L = 0;
      pd1 = (unsigned long long)((slot_in[d.r1] ? p.pop1 : p.pop0) + (size_t)d.r1 * p.pitch);
      pd2 = (unsigned long long)((slot_in[d.r2] ? p.pop1 : p.pop0) + (size_t)d.r2 * p.pitch);
      pd3 = (unsigned long long)((slot_in[d.r3] ? p.pop1 : p.pop0) + (size_t)d.r3 * p.pitch);
    }
    const int jrand = __shfl_sync(0xFFFFFFFFu, d.jrand, 0);
    const int L = __shfl_sync(0xFFFFFFFFu, d.L, 0);
    const float4* d1 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd1, 0));
    const float4* d2 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd2, 0));
    const float4* d3 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd3, 0));
    int cnt = 0;
    float nrm = 0.0f, amx = 0.0f;
    for (int q0 = 0; q0 < p.D4; q0 += 32 * kTrialUnroll) {
      if (q0 > 0) {
#pragma unroll
        for (int u = 0; u < kTrialUnroll; ++u) {
          const int q = q0 + lane + 32 * u;
          x[u] = (q < p.D4) ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
      }
#pragma unroll
      for (int u = 0; u < kTrialUnroll; ++u) {
        const int q = q0 + lane + 32 * u;
        if (q >= p.D4) continue;
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
          if (dd < 0) dd += p.D;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            int de = dd + e;
            if (de >= p.D) de -= p.D;
            m |= (de < L) ? (1u << e) : 0u;
          }
        }
        m &= (1u << min(4, p.D - j0)) - 1u;
        float4 v = x[u];
        if (m) {
          const float4 a1 = ld_ro(d1 + q), a2 = ld_ro(d2 + q), a3 = ld_ro(d3 + q);
          mutate_slot(v, a1, a2, a3, m, p);
        }
        if constexpr (XO == kBin) cnt += __popc(m);
        st_stream(trow + q, v);
        if (p.dbg_trial) reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * p.pitch)[q] = v;
        float a[4];
        if (j0 + 4 <= p.D) {                       // a full slot: o by one 16-byte load
          const float4 o4 = __ldg(reinterpret_cast<const float4*>(sp.shift) + q);
          a[0] = __fsub_rn(v.x, o4.x);
          a[1] = __fsub_rn(v.y, o4.y);
          a[2] = __fsub_rn(v.z, o4.z);
          a[3] = __fsub_rn(v.w, o4.w);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = j0 + e;
            a[e] = (j < p.D) ? __fsub_rn(lane_of(v, e), sp.shift[j]) : 0.0f;
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          nrm = fmaf(a[e], a[e], nrm);
          amx = fmaxf(amx, fabsf(a[e]));
        }
        if (sp.prec != 0) {                        // D % 256 == 0 on this path: 8-byte aligned
          uint32_t h[4], l[4];
          if (sp.prec == 3) {                      // FP16 halves of 2^sa a (the scaling is exact)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float as = a[e] * sp.a_scale;
              const __half hi = __float2half_rn(as);
              const __half lo = __float2half_rn(__fsub_rn(as, __half2float(hi)));
              h[e] = __half_as_ushort(hi);
              l[e] = __half_as_ushort(lo);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(a[e]);
              const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(a[e], __bfloat162float(hi)));
              h[e] = __bfloat16_as_ushort(hi);
              l[e] = __bfloat16_as_ushort(lo);
            }
          }
          *reinterpret_cast<uint2*>(sp.a_hi + (size_t)i * p.D + j0) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
          *reinterpret_cast<uint2*>(sp.a_lo + (size_t)i * p.D + j0) = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm += __shfl_xor_sync(0xFFFFFFFFu, nrm, o);
      amx = fmaxf(amx, __shfl_xor_sync(0xFFFFFFFFu, amx, o));
      cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
    Lrow = (XO == kBin) ? cnt : L;
    if (lane == 0) {
      sp.norm2[i] = nrm;
      sp.amax[i] = amx;
      if (p.dbg_draws) {
        int* o = p.dbg_draws + 5 * (size_t)i;
        o[0] = d.r1; o[1] = d.r2; o[2] = d.r3; o[3] = d.jrand; o[4] = Lrow;
      }
    }
  }
  if (lane == 0) wcnt[warp] = Lrow;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long c = 0;
    for (int w = 0; w < kTrialWarps; ++w) c += (unsigned long long)wcnt[w];
    atomicAdd(&p.st->masked, c);
  }
}

// ---------------------------------------------------------------------------
// FP32 product with the fitness epilogue
// mode 0: all rows, trial rows (other slot); 1: all rows, parent rows;
// 2: the ambiguous entries (row << 1 | parent flag), partials to part2_*.
//
// Every z_ik is one FMA chain over j ascending (zero padding past D adds
// fma(0, 0, acc) = acc), and every 64-column partial sums g over the column
// tile the same way in both kernels below: each of 16 lanes adds its 4
// consecutive columns in order, then an xor tree over the 16 lanes
// (offsets 8, 4, 2, 1). So a row's partials do not depend on the kernel, the
// tile or the other rows: the re-evaluation kernel reproduces the all-rows
// kernel bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ const float* sr_row_ptr(const SrParams& sp, int mode, int e, const uint8_t* slot_in) {
  const GenParams& p = sp.g;
  int r = e, parent = (mode == 1);
  if (mode == 2) {
    r = sp.amb[e] >> 1;
    parent = sp.amb[e] & 1;
  }
  const int s = slot_in[r];
  const int buf = parent ? s : 1 - s;
  return (buf ? p.pop1 : p.pop0) + (size_t)r * p.pitch;
}

// One row's 4 columns of a 64-column tile, reduced over the tile's 16 lanes
// (all 32 lanes of the warp call it; lanes 16..31 reduce their own tile row).
__device__ __forceinline__ void sr_tile_reduce(const SrParams& sp, const float z[4], int c0, float& sg, float& sw) {
  const GenParams& p = sp.g;
  sg = 0.0f;
  sw = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int n = c0 + b;
    if (n < p.D) {
      const float w = sr_weight(sp.obj, n, p.ell_k);
      sg += sr_g(sp.obj, z[b], w);
      sw = fmaf(w, fabsf(z[b]), sw);
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    sg += __shfl_xor_sync(0xFFFFFFFFu, sg, o);
    sw += __shfl_xor_sync(0xFFFFFFFFu, sw, o);
  }
}

// All rows (modes 0 and 1): 128 x 128 output tile, 256 threads, 8 rows x
// (2 x 4) columns per thread (columns tx*4.. and 64 + tx*4.. so that each
// 64-column half keeps the lane layout above), K in steps of 16 through a
// double-buffered shared-memory stage with the next step prefetched into
// registers. VEC: D % 4 == 0, 16-byte loads of x, o and R.
constexpr int kGbM = 128, kGbN = 128, kGbK = 16, kGbLd = kGbM + 4;

template <bool VEC>
__global__ void __launch_bounds__(256, 2) sr_gemm_fp32_kernel(const __grid_constant__ SrParams sp, int mode) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  __shared__ __align__(16) float As[2][kGbK][kGbLd];
  __shared__ __align__(16) float Bs[2][kGbK][kGbLd];
  __shared__ const float* rowp[kGbM];

  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int n0 = blockIdx.x * kGbN, r0 = blockIdx.y * kGbM;
  const long long gen = p.st->gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  if (t < kGbM) rowp[t] = (r0 + t < p.N) ? sr_row_ptr(sp, mode, r0 + t, slot_in) : nullptr;
  __syncthreads();

  // loader: row / column lm of the tile, 8 consecutive k from lk
  const int lm = t & (kGbM - 1), lk = (t >> 7) * 8;
  const float* xa = rowp[lm];
  const float* rb = (n0 + lm < p.D) ? sp.rot + (size_t)(n0 + lm) * p.D : nullptr;
  float va[8], vb[8];
  auto load = [&](int k0) {
    const int j0 = k0 + lk;
    if constexpr (VEC) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = j0 + 4 * h;
        float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), r4 = x4;
        if (j < p.D) {
          const float4 o4 = *reinterpret_cast<const float4*>(sp.shift + j);
          if (xa) {
            x4 = *reinterpret_cast<const float4*>(xa + j);
            x4 = make_float4(__fsub_rn(x4.x, o4.x), __fsub_rn(x4.y, o4.y), __fsub_rn(x4.z, o4.z), __fsub_rn(x4.w, o4.w));
          }
          if (rb) r4 = *reinterpret_cast<const float4*>(rb + j);
        }
        va[4 * h + 0] = x4.x; va[4 * h + 1] = x4.y; va[4 * h + 2] = x4.z; va[4 * h + 3] = x4.w;
        vb[4 * h + 0] = r4.x; vb[4 * h + 1] = r4.y; vb[4 * h + 2] = r4.z; vb[4 * h + 3] = r4.w;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        va[u] = (xa && j < p.D) ? __fsub_rn(xa[j], sp.shift[j]) : 0.0f;
        vb[u] = (rb && j < p.D) ? rb[j] : 0.0f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      As[buf][lk + u][lm] = va[u];
      Bs[buf][lk + u][lm] = vb[u];
    }
  };

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;

  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < p.D; k0 += kGbK) {
    const bool more = k0 + kGbK < p.D;
    if (more) load(k0 + kGbK);
#pragma unroll
    for (int kk = 0; kk < kGbK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(ar[a], br[b], acc[a][b]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  float* pg = sp.part_g;
  float* pw = sp.part_w;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int e = r0 + ty * 8 + a;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float z[4] = {acc[a][4 * h], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]};
      const int c0 = n0 + 64 * h;
      float sg, sw;
      sr_tile_reduce(sp, z, c0 + tx * 4, sg, sw);
      if (tx == 0 && e < p.N && c0 < p.D) {
        pg[(size_t)e * sp.nct2 + (c0 >> 6)] = sg;
        pw[(size_t)e * sp.nct2 + (c0 >> 6)] = sw;
      }
    }
  }
}

// The ambiguous entries (mode 2; split-operand paths only, so D % 256 == 0):
// work items of 16 entries x 64 columns, taken by groups of 4 warps (2
// entries x 4 columns per lane: lanes 0-15 take entries 0-1 of the warp, lanes
// 16-31 entries 2-3, and lane tx = lane & 15 columns 4 tx .. 4 tx + 3 of the
// 64-column tile, the layout the tile reduction expects). Each group has its
// own 4-stage cp.async ring of 64-deep slices of the entries' rows of x, o
// and rows of R^T (three stages in flight cover the L2 latency of the short
// per-stage work) and its own named barrier. Once a stage has landed, each
// warp forms a = fl(x - o) K-major for its own four entries (so only a warp
// barrier follows), and the inner loop is an 8-byte and a 16-byte shared load
// and eight FMAs per k: every z stays one FMA chain over j ascending. The list is
// short (a few hundred entries) and each chain is D FMAs long, so the time is
// set by the busiest SM. Two groups per CTA and a ring per group that needs
// more than half an SM's shared memory for the pair put exactly one CTA on
// each SM; the grid is one CTA per SM, group g of CTA b takes items
// b + g * grid, b + (2 + g) * grid, ..., so the first items of a short list
// land on distinct SMs whatever order the CTAs are placed in.
constexpr int kLsE = 16, kLsN = 64, kLsK = 64, kLsStages = 4, kLsGroupThreads = 128, kLsGroups = 2;
constexpr int kLsThreads = kLsGroups * kLsGroupThreads;
constexpr int kLsLdX = kLsK + 4, kLsLdB = kLsN + 4, kLsLdA = kLsE + 4;   // floats per row
constexpr int kLsGroupFloats = kLsStages * (kLsE * kLsLdX + kLsK + kLsK * kLsLdB) + kLsK * kLsLdA;
constexpr size_t kLsSmem = sizeof(float) * (size_t)kLsGroups * kLsGroupFloats;
static_assert(kLsSmem > 114 * 1024 && kLsSmem <= 227 * 1024, "one CTA per SM");

__device__ __forceinline__ void ls_group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kLsGroupThreads) : "memory");
}

__global__ void __launch_bounds__(kLsThreads, 1) sr_gemm_fp32_list_kernel(const __grid_constant__ SrParams sp) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  extern __shared__ __align__(16) float ls_smem[];
  const int g = threadIdx.x / kLsGroupThreads, t = threadIdx.x % kLsGroupThreads;
  float* Xs = ls_smem + (size_t)g * kLsGroupFloats;  // [stage][entry][kLsLdX]: raw x
  float* Os = Xs + kLsStages * kLsE * kLsLdX;      // [stage][k]: o
  float* Bs = Os + kLsStages * kLsK;               // [stage][k][kLsLdB]: R^T rows
  float* As = Bs + kLsStages * kLsK * kLsLdB;      // [k][kLsLdA]: a per entry
  __shared__ const float* rowp_all[kLsGroups][kLsE];
  const float** rowp = rowp_all[g];
  const int lane = t & 31, warp = t >> 5;
  const int tx = lane & 15;
  const int ebase = warp * 4 + (lane >> 4) * 2;    // the lane's first entry in the tile
  const long long gen = p.st->gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  const int nrows = (int)*sp.amb_count;
  const int KS = p.D / kLsK, ctiles = p.D / kLsN;
  const int items = ((nrows + kLsE - 1) / kLsE) * ctiles;
  int n0 = 0;

  // one stage: x 16 entries x 16 chunks of 16 bytes (two per thread), o 16
  // chunks, R^T 64 rows x 16 chunks (8 per thread); entries past the list
  // read zeros
  auto issue = [&](int step) {
    const int st = step % kLsStages, k0 = step * kLsK;
#pragma unroll
    for (int i = 0; i < (kLsE * kLsK / 4) / kLsGroupThreads; ++i) {
      const int qx = t + kLsGroupThreads * i, m = qx / (kLsK / 4), c = (qx % (kLsK / 4)) * 4;
      const float* xa = rowp[m];
      cp_async16(sr_smem_u32(Xs + (st * kLsE + m) * kLsLdX + c), xa ? xa + k0 + c : sp.shift, xa ? 16u : 0u);
    }
    if (t < kLsK / 4) cp_async16(sr_smem_u32(Os + st * kLsK + 4 * t), sp.shift + k0 + 4 * t, 16u);
#pragma unroll
    for (int i = 0; i < (kLsK * kLsN / 4) / kLsGroupThreads; ++i) {
      const int q = t + kLsGroupThreads * i, kr = q >> 4, c = (q & 15) * 4;
      cp_async16(sr_smem_u32(Bs + (st * kLsK + kr) * kLsLdB + c), sp.rot_t + (size_t)(k0 + kr) * p.D + n0 + c, 16u);
    }
  };

  for (int item = blockIdx.x + g * gridDim.x; item < items; item += kLsGroups * gridDim.x) {
    const int r0 = (item / ctiles) * kLsE, ct = item % ctiles;
    n0 = ct * kLsN;
    ls_group_sync(g);                              // rowp and the stages are reused
    if (t < kLsE) rowp[t] = (r0 + t < nrows) ? sr_row_ptr(sp, 2, r0 + t, slot_in) : nullptr;
    ls_group_sync(g);
#pragma unroll
    for (int s0 = 0; s0 < kLsStages - 1; ++s0) {
      if (s0 < KS) issue(s0);
      cp_async_commit();
    }
    float acc[2][4];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[e][c] = 0.0f;
    for (int step = 0; step < KS; ++step) {
      cp_async_wait<kLsStages - 2>();
      ls_group_sync(g);                             // this stage landed; every lane is done with the
                                                    // slot refilled next
      if (step + kLsStages - 1 < KS) issue(step + kLsStages - 1);
      cp_async_commit();
      const int st = step % kLsStages;
#pragma unroll
      for (int kk = lane; kk < kLsK; kk += 32) {   // a = fl(x - o): k = kk, the warp's 4 entries
        const int m0 = warp * 4;
        const float* xs = Xs + (st * kLsE + m0) * kLsLdX + kk;
        const float o = Os[st * kLsK + kk];
        *reinterpret_cast<float4*>(As + kk * kLsLdA + m0) =
            make_float4(__fsub_rn(xs[0], o), __fsub_rn(xs[kLsLdX], o), __fsub_rn(xs[2 * kLsLdX], o),
                        __fsub_rn(xs[3 * kLsLdX], o));
      }
      __syncwarp();                                 // a of the warp's entries, written by the warp
      const float* as = As + ebase;
      const float* bs = Bs + st * kLsK * kLsLdB + 4 * tx;
#pragma unroll
      for (int k = 0; k < kLsK; ++k) {
        const float2 av = *reinterpret_cast<const float2*>(as + k * kLsLdA);
        const float4 bv = *reinterpret_cast<const float4*>(bs + k * kLsLdB);
        acc[0][0] = fmaf(av.x, bv.x, acc[0][0]);
        acc[0][1] = fmaf(av.x, bv.y, acc[0][1]);
        acc[0][2] = fmaf(av.x, bv.z, acc[0][2]);
        acc[0][3] = fmaf(av.x, bv.w, acc[0][3]);
        acc[1][0] = fmaf(av.y, bv.x, acc[1][0]);
        acc[1][1] = fmaf(av.y, bv.y, acc[1][1]);
        acc[1][2] = fmaf(av.y, bv.z, acc[1][2]);
        acc[1][3] = fmaf(av.y, bv.w, acc[1][3]);
      }
    }                                               // (the next step's group barrier orders the As reuse)
    cp_async_wait<0>();
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int ent = r0 + ebase + e;
      float sg, sw;
      sr_tile_reduce(sp, acc[e], n0 + 4 * tx, sg, sw);
      if (tx == 0 && ent < nrows) {
        sp.part2_g[(size_t)ent * sp.nct2 + ct] = sg;
        sp.part2_w[(size_t)ent * sp.nct2 + ct] = sw;
      }
    }
  }
}

cudaError_t prepare_sr_list(int* ctas) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *ctas = sms > 0 ? sms : 1;
  return cudaFuncSetAttribute(sr_gemm_fp32_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLsSmem);
}

// R^T for the list kernel's contiguous B tiles (once, at set-up).
__global__ void sr_transpose_kernel(const float* __restrict__ rot, float* __restrict__ rot_t, int D) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = by + r, j = bx + threadIdx.x;
    tile[r][threadIdx.x] = (k < D && j < D) ? rot[(size_t)k * D + j] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = bx + r, k = by + threadIdx.x;
    if (j < D && k < D) rot_t[(size_t)j * D + k] = tile[threadIdx.x][r];
  }
}

cudaError_t launch_sr_transpose(const float* rot, float* rot_t, int D, cudaStream_t s) {
  const dim3 grid((unsigned)((D + 31) / 32), (unsigned)((D + 31) / 32)), blk(32, 8);
  sr_transpose_kernel<<<grid, blk, 0, s>>>(rot, rot_t, D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// decisions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sr_row_value(const float* pg, int nct) {
  float f = 0.0f;
  for (int c = 0; c < nct; ++c) f += pg[c];
  return (f != f) ? __int_as_float(0x7F800000) : f;
}

// Bound on |f_split - f_FP32path| of one row (BF16 or FP16 split operands)
// from n^2 = |a|_2^2, the row's sum_k w_k |z_k| and its value f.
// Worst case: |dz_k| <= delta = c n + delta_abs for every k; Rastrigin |dg| <=
// delta (2|z| + 20 pi + 3 delta); elliptic |dg_k| <= w_k delta (2|z_k| +
// delta); plus the reductions' relative error.
// Probabilistic: the first-order change sum_k g'(z_k) dz_k is a sum of
// independent zero-mean terms (operand-split residuals, accumulation
// roundings) whose bounds give the standard deviations; the g evaluations and
// the sums over k add theirs (tsq: the sum of the squares of the row's tile
// partials). The tensor cores' FP32 accumulator rounds toward zero, which
// shrinks every |z_k| a little: half an ulp, at most 2^-24 |z_k|, per MMA step
// of the leading product on average bounds that bias, and the correction
// products' steps, on partial sums ~2 u_s smaller, add a term in n H.
// Second-order terms are bounded by the mean of |dz|_2^2 with a factor 2.
__device__ __forceinline__ float sr_bound(int obj, float norm2, float amax, float sumw, float f, float tsq, int D,
                                         const SrBound& b) {
  if (b.mode == 1) {
    const float delta = b.delta_per_norm * sqrtf(norm2) * 1.0001f + b.delta_abs;
    float e;
    if (obj == kSrElliptic) e = delta * (2.0f * sumw + delta * b.sum_w);
    else e = delta * (2.0f * sumw + (float)D * (20.0f * 3.14159274f + 3.0f * delta));
    return (e + b.rel * fabsf(f)) * 1.001f;
  }
  const float n = sqrtf(norm2) * 1.0001f;
  const float af = fabsf(f);
  // |g'(z)| for Rastrigin: 2|z| + 20 pi |sin 2 pi z| <= min(2|z| + 20 pi, (2 + 40 pi^2) |z|)
  const float H = (obj == kSrElliptic) ? 2.0f * sqrtf(b.wmax * af * 1.0001f)
                                       : fminf(2.0002f * n + b.hconst, 396.7843f * n);
  const float rep = fmaf(b.rep_k, amax * 1.0001f, b.rep_f);
  const float s_rep = 1.7320509f * rep * H, s_acc = b.acc_c * n * H;
  const float s_ev = b.eval_c * af + b.sum_u * sqrtf(b.sum_f2 * af * af + b.sum_t2 * tsq);
  const float sig = sqrtf(s_rep * s_rep + s_acc * s_acc + s_ev * s_ev);
  const float bias = b.bias_c * ((obj == kSrElliptic) ? 2.0f * af : n * H) + b.bias_c2 * n * H;
  // A row with a = 0 exactly has z = 0 exactly on both paths: B = 0. Any other
  // row keeps a floor, so that terms underflowing in FP32 never leave B = 0.
  const float B = (b.lambda * sig + bias + b.quad_a * rep * rep + b.quad_b * norm2) * 1.001f;
  return amax > 0.0f ? fmaxf(B, 1e-36f) : B;
}

// Warp-aggregated updates of the generation's counters: one atomic per warp
// instead of one per row (every lane of the warp calls these).
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ void warp_note_accepts(DevState* st, bool acc, unsigned long long key) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, acc);
  if (m == 0u) return;                             // uniform across the warp
  const unsigned long long k = warp_min_u64(acc ? key : ~0ull);
  if ((threadIdx.x & 31) == __ffs(m) - 1) {
    atomicMin(&st->best_key, k);
    atomicAdd(&st->accepts, (unsigned long long)__popc(m));
  }
}

// One row per thread (the grid covers N once).
__global__ void sr_select_kernel(const __grid_constant__ SrParams sp, SrBound bnd) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  const long long gen = p.st->gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (i == 0) *sp.finish_due = (sp.inc_every > 0 && (gen + 1) % sp.inc_every == 0) ? 1 : 0;
  int decision = 0;                                // 1 accept, 0 reject, 2 ambiguous
  float f = 0.0f, bx = 0.0f;
  if (i < p.N) {
    const int si = slot_in[i];
    f = sr_row_value(sp.part_g + (size_t)i * sp.nct, sp.nct);
    float bu = 0.0f;
    if (sp.prec != 0) {
      float sw = 0.0f, tsq = 0.0f;                 // sum of the tile partials' squares
      for (int c = 0; c < sp.nct; ++c) {
        const float t = sp.part_g[(size_t)i * sp.nct + c];
        tsq = fmaf(t, t, tsq);
      }
      if (bnd.mode == 1)
        for (int c = 0; c < sp.nct; ++c) sw += sp.part_w[(size_t)i * sp.nct + c];
      bu = sr_bound(sp.obj, sp.norm2[i], sp.amax[i], sw, f, tsq * 1.0001f, p.D, bnd);
    }
    const float fx = p.fit[i];
    bx = sp.fit_err[i];
    if (bu == 0.0f && bx == 0.0f) decision = (f < fx) ? 1 : 0;
    else if (f + bu < fx - bx) decision = 1;
    else if (f - bu >= fx + bx) decision = 0;
    else decision = 2;
    if (decision == 1) {
      slot_out[i] = (uint8_t)(1 - si);
      p.fit[i] = f;
      sp.fit_err[i] = bu;
    } else {
      slot_out[i] = (uint8_t)si;
    }
    if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
    if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)(decision == 1);
  }
  warp_note_accepts(p.st, decision == 1, best_key_of(f, i));
  // ambiguous rows: the trial, and the parent when its stored value is inexact,
  // in consecutive entries; one reservation per warp
  const unsigned need = (decision == 2) ? (bx > 0.0f ? 2u : 1u) : 0u;
  unsigned incl = need;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  if (total > 0u) {                                // uniform across the warp
    const unsigned rows = __popc(__ballot_sync(0xFFFFFFFFu, need > 0u));
    unsigned base = 0u;
    if (lane == 31) {
      base = atomicAdd(sp.amb_count, total);
      atomicAdd(&p.st->reselected, (unsigned long long)rows);
    }
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    if (need > 0u) {
      const unsigned k = base + incl - need;
      sp.amb[k] = i << 1;                          // the trial
      if (need == 2u) sp.amb[k + 1] = (i << 1) | 1;  // and the parent
    }
  }
}

// Ambiguous rows: decide with FP32-path values of the trial (and the parent).
// One entry per thread (the grid covers 2N entries once).
__global__ void sr_resolve_kernel(const __grid_constant__ SrParams sp) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  const long long gen = p.st->gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  const unsigned n = *sp.amb_count;
  const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x >= n) return;        // uniform across the CTA
  bool acc = false;
  float fu = 0.0f;
  int i = 0;
  if (e < n && !(sp.amb[e] & 1)) {                 // parents are read by their trial's entry
    i = sp.amb[e] >> 1;
    fu = sr_row_value(sp.part2_g + (size_t)e * sp.nct2, sp.nct2);
    float fx = p.fit[i];
    if (e + 1 < n && sp.amb[e + 1] == ((i << 1) | 1)) {
      fx = sr_row_value(sp.part2_g + (size_t)(e + 1) * sp.nct2, sp.nct2);
      p.fit[i] = fx;                               // the parent's exact FP32-path value
      sp.fit_err[i] = 0.0f;
    }
    const int si = slot_in[i];
    acc = fu < fx;
    if (acc) {
      slot_out[i] = (uint8_t)(1 - si);
      p.fit[i] = fu;
      sp.fit_err[i] = 0.0f;
    }
    if (p.dbg_ftrial) p.dbg_ftrial[i] = fu;
    if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
  }
  warp_note_accepts(p.st, acc, best_key_of(fu, i));
}

// Initial evaluation (always the FP32 product, whose partials have nct2
// columns): fit = sum of partials, fit_err = 0, best key.
__global__ void sr_store_eval_kernel(const __grid_constant__ SrParams sp) {
  const GenParams& p = sp.g;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x) {
    const float f = sr_row_value(sp.part_g + (size_t)i * sp.nct2, sp.nct2);
    p.fit[i] = f;
    sp.fit_err[i] = 0.0f;
    atomicMin(&p.st->best_key, best_key_of(f, i));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_sr_trial(int xo, int /*vidx*/, const SrParams& sp, int /*block*/, cudaStream_t s) {
  const unsigned grid = (unsigned)((sp.g.N + kTrialWarps - 1) / kTrialWarps);
  if (xo == kBin) return launch_pdl(sr_trial_kernel<kBin>, dim3(grid), dim3(kTrialWarps * 32), 0, s, sp);
  if (xo == kExp) return launch_pdl(sr_trial_kernel<kExp>, dim3(grid), dim3(kTrialWarps * 32), 0, s, sp);
  return launch_pdl(sr_trial_kernel<kNec>, dim3(grid), dim3(kTrialWarps * 32), 0, s, sp);
}

cudaError_t launch_sr_gemm_fp32(const SrParams& sp, int mode, int max_rows, cudaStream_t s) {
  const unsigned gx = (unsigned)((sp.g.D + kGbN - 1) / kGbN);
  if (mode == 2) {                                // split-operand paths: D % 256 == 0
    if (sp.g.D % kLsN != 0) return cudaErrorInvalidValue;
    const int items = ((max_rows + kLsE - 1) / kLsE) * (sp.g.D / kLsN);
    const int grid = std::max(1, std::min(sp.list_ctas, (items + kLsGroups - 1) / kLsGroups));
    return launch_pdl(sr_gemm_fp32_list_kernel, dim3((unsigned)grid), dim3(kLsThreads), kLsSmem, s, sp);
  }
  const dim3 grid(gx, (unsigned)((max_rows + kGbM - 1) / kGbM));
  if (sp.g.D % 4 == 0) return launch_pdl(sr_gemm_fp32_kernel<true>, grid, dim3(256), 0, s, sp, mode);
  return launch_pdl(sr_gemm_fp32_kernel<false>, grid, dim3(256), 0, s, sp, mode);
}

cudaError_t launch_sr_select(const SrParams& sp, const SrBound& b, cudaStream_t s) {
  return launch_pdl(sr_select_kernel, dim3((sp.g.N + 255) / 256), dim3(256), 0, s, sp, b);
}

cudaError_t launch_sr_resolve(const SrParams& sp, cudaStream_t s) {
  return launch_pdl(sr_resolve_kernel, dim3((2 * sp.g.N + 255) / 256), dim3(256), 0, s, sp);
}

cudaError_t launch_sr_store_eval(const SrParams& sp, cudaStream_t s) {
  sr_store_eval_kernel<<<(sp.g.N + 255) / 256, 256, 0, s>>>(sp);
  return cudaGetLastError();
}

}  // namespace de

namespace de {

// R -> hi(R), lo(R) = the rounded remainder: BF16 halves of R, or FP16
// halves of 2^sr R (scale = 2^sr, exact).
__global__ void sr_split_kernel(const float* rot, uint16_t* hi, uint16_t* lo, size_t n, int fp16, float scale) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const float r = rot[k];
    if (fp16) {
      const float rs = r * scale;
      const __half h = __float2half_rn(rs);
      hi[k] = __half_as_ushort(h);
      lo[k] = __half_as_ushort(__float2half_rn(__fsub_rn(rs, __half2float(h))));
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      hi[k] = __bfloat16_as_ushort(h);
      lo[k] = __bfloat16_as_ushort(__float2bfloat16_rn(__fsub_rn(r, __bfloat162float(h))));
    }
  }
}

cudaError_t launch_sr_split_rotation(const float* rot, uint16_t* hi, uint16_t* lo, size_t n, bool fp16, float scale,
                                     cudaStream_t s) {
  sr_split_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(rot, hi, lo, n, fp16 ? 1 : 0,
                                                                                     scale);
  return cudaGetLastError();
}

// The incumbent in FP64 (the only FP64 arithmetic on the GPU), fused with
// the close of the generation. Generation g' = g + 1 when closing (g itself
// for the initial evaluation); every `every` generations the best row's
// objective is recomputed as z = R (x - o) and sum g(z) in FP64: one warp per
// z_k (coalesced reads of row k of R, lanes over j, a fixed shuffle tree),
// g(z_k) to inc_part[k]. The last CTA to finish (a ticket) sums inc_part in a
// fixed order, so the value does not depend on scheduling, and then closes
// the generation: best value and generation, the counter, the ambiguous list.
// Every CTA reads the state before it takes its ticket, and only the last
// one writes it.
constexpr int kIncWarps = 8;

// The close of a generation: best value and its generation, the counter, the
// base row of the next generation, an empty ambiguous list.
__device__ __forceinline__ void sr_close_generation(DevState* st, long long gnext, unsigned* amb_count) {
  const float bf = from_ordered_bits((uint32_t)(st->best_key >> 32));
  if (bf < st->best_f) {
    st->best_f = bf;
    st->best_gen = gnext;
  }
  st->gen = gnext;
  st->base_row = (int)(uint32_t)(st->best_key & 0xFFFFFFFFull);
  *amb_count = 0u;
}

__global__ void __launch_bounds__(kIncWarps * 32) sr_finish_kernel(const __grid_constant__ SrParams sp, int every,
                                                                  int close) {
  griddep_wait();                                  // the previous kernel of the generation is done
  griddep_launch_dependents();
  const GenParams& p = sp.g;
  // Closing a generation: whether the incumbent is due was recorded by this
  // generation's selection kernel, so that CTA 0 may close the generation
  // (write the counter) alone while the other CTAs are still deciding.
  // Without a close nothing writes the counter.
  const bool due = close ? (*sp.finish_due != 0) : (every > 0 && p.st->gen % every == 0);
  if (!due && !close) return;                       // uniform across the grid
  if (!due) {                                       // nothing to re-evaluate: CTA 0 closes alone
    if (blockIdx.x == 0 && threadIdx.x == 0) sr_close_generation(p.st, p.st->gen + 1, sp.amb_count);
    return;
  }
  const long long gen = p.st->gen;                  // written only by the last CTA below
  const long long gnext = close ? gen + 1 : gen;
  const int idx = (int)(uint32_t)(p.st->best_key & 0xFFFFFFFFull);
  const bool have = due && idx >= 0 && idx < p.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (have) {
    const int si = p.slots[(size_t)(gnext & 1) * p.N + idx];
    const float* x = (si ? p.pop1 : p.pop0) + (size_t)idx * p.pitch;
    const int k = blockIdx.x * kIncWarps + warp;
    if (k < p.D) {
      const float* r = sp.rot + (size_t)k * p.D;
      double z = 0.0;
      for (int j = lane; j < p.D; j += 32) z = fma((double)r[j], (double)x[j] - (double)sp.shift[j], z);
      for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xFFFFFFFFu, z, o);
      if (lane == 0) {
        double gk;
        if (sp.obj == kSrElliptic) {
          const double c = (p.D > 1) ? exp2((double)k * (6.0 * 3.321928094887362 / (double)(p.D - 1))) : 1.0;
          gk = c * z * z;
        } else {
          gk = z * z - 10.0 * cos(2.0 * 3.141592653589793 * z) + 10.0;
        }
        sp.inc_part[k] = gk;
      }
    }
  }
  __shared__ unsigned ticket;
  __shared__ double red[kIncWarps * 32];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(sp.inc_count, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  if (have) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < p.D; q += blockDim.x) acc += __ldcg(sp.inc_part + q);
    red[threadIdx.x] = acc;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (have) {
      double f = 0.0;
      for (int w = 0; w < (int)blockDim.x; ++w) f += red[w];
      p.st->incumbent_f64 = f;
      p.st->incumbent_gen = gnext;
    }
    if (close) sr_close_generation(p.st, gnext, sp.amb_count);
    *sp.inc_count = 0u;
  }
}

cudaError_t launch_sr_finish(const SrParams& sp, int every, bool close, cudaStream_t s) {
  const unsigned grid = (unsigned)((sp.g.D + kIncWarps - 1) / kIncWarps);
  return launch_pdl(sr_finish_kernel, dim3(grid), dim3(kIncWarps * 32), 0, s, sp, every, close ? 1 : 0);
}

}  // namespace de
