// batch_span.cuh — the row kernel of the batched generation for instances
// whose rows take at most one warp (G = 4, 8, 16 or 32 lanes per row, at
// most 16 float4 slots per lane).
//
// Work is a list of spans, each up to 32 consecutive rows of one instance,
// grouped by (objective, crossover, G) so that one specialisation of the row
// code runs at a time. Warps take spans from a global queue (one atomic per
// span, so long and short spans balance themselves). At the start of a span
// the warp stages the span's row plans (donors, j_rand, L, slot bytes, parent
// fitness: 32 bytes each) in shared memory with one coalesced load and reads
// the instance's parameters once; each row then costs one memory round trip
// (the parent row and the donor genes of its masked slots, issued together).
//
// Reduction order. The FP32 fitness of a row is summed in an order that does
// not depend on G: 32 virtual lanes v, virtual lane v summing the genes of
// the float4 slots q = v, v + 32, v + 64, ... in ascending gene order, then a
// butterfly over v with strides 16, 8, 4, 2, 1. A lane of a G-lane group
// holds the virtual lanes gl + G t (t < 32 / G) in separate accumulators, so
// the strides >= G are additions inside the lane and the smaller ones are
// shuffles. Every choice of G therefore gives bit-identical fitness values,
// selections and trajectories, and the tile shape can be tuned freely.
#pragma once
#include "draws.cuh"
#include "internal.h"
#include "objectives.cuh"

namespace de {

constexpr int kSpanThreads = 256;
constexpr int kSpanVmax = 16;

// The rows [row0, row0 + rows) of one instance, R = 32 / G rows at a time.
// spl: the span's plans in shared memory (unused when eval_only).
template <int OBJ, int XO, int G>
__device__ __noinline__ void span_rows(const BatchInst* __restrict__ Ip, int row0, int rows,
                                       const RowPlan32* spl, int eval_only) {
  constexpr int R = 32 / G;                       // rows per warp pass = accumulator sets per lane
  constexpr int NS = ObjTraits<OBJ>::kSums;
  const GenParams& p = Ip->g;
  const int lane = threadIdx.x & 31;
  const int gi = lane / G, gl = lane % G;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const int D = p.D, D4 = p.D4, N = p.N;
  const size_t pitch = (size_t)p.pitch;
  const float F = p.F, lo = p.lo, hi = p.hi;
  const float* pop0 = p.pop0;
  const float* pop1 = p.pop1;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * N;

  unsigned long long kmin = ~0ull, masked_sum = 0ull;
  unsigned accepts = 0u;

  for (int r = 0; r < rows; r += R) {
    const int li = r + gi;
    const bool active = li < rows;
    const int i = row0 + (active ? li : 0);
    RowPlan32 pl;
    if (eval_only) {
      pl.r1 = pl.r2 = pl.r3 = 0;
      pl.jrand = 0;
      pl.L = 0;
      pl.fit_i = 0.0f;
      pl.slots = active ? (uint32_t)slot_in[i] : 0u;
    } else {
      pl = spl[active ? li : 0];
    }
    const int si = (int)(pl.slots & 0xFFu);
    const float4* xrow = reinterpret_cast<const float4*>((si ? pop1 : pop0) + (size_t)i * pitch);
    const float4* d1 = reinterpret_cast<const float4*>(((pl.slots >> 8) & 0xFFu ? pop1 : pop0) + (size_t)pl.r1 * pitch);
    const float4* d2 = reinterpret_cast<const float4*>(((pl.slots >> 16) & 0xFFu ? pop1 : pop0) + (size_t)pl.r2 * pitch);
    const float4* d3 = reinterpret_cast<const float4*>(((pl.slots >> 24) & 0xFFu ? pop1 : pop0) + (size_t)pl.r3 * pitch);

    // parent slots and crossover masks (4 bits per slot)
    float4 x[kSpanVmax];
    unsigned long long mks = 0ull;
#pragma unroll
    for (int k = 0; k < kSpanVmax; ++k) {
      const int q = gl + k * G;
      const bool in = active && q < D4;
      x[k] = in ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      unsigned m = 0u;
      if (in && !eval_only) {
        const int j0 = 4 * q;
        if constexpr (XO == kBin) {
          const uint4 w = philox_block(p.key, kStreamBin, p.inst, g, (uint32_t)i, (uint32_t)q);
          m |= ((unsigned long long)w.x < p.cr_t || j0 + 0 == pl.jrand) ? 1u : 0u;
          m |= ((unsigned long long)w.y < p.cr_t || j0 + 1 == pl.jrand) ? 2u : 0u;
          m |= ((unsigned long long)w.z < p.cr_t || j0 + 2 == pl.jrand) ? 4u : 0u;
          m |= ((unsigned long long)w.w < p.cr_t || j0 + 3 == pl.jrand) ? 8u : 0u;
        } else {
          int dd = j0 - pl.jrand;
          if (dd < 0) dd += D;                     // (j0 - j_rand) mod D
          if (!(dd >= pl.L && dd + 3 < D)) {       // some gene of the slot may lie in the segment
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              int de = dd + e;
              if (de >= D) de -= D;
              m |= (de < pl.L) ? (1u << e) : 0u;
            }
          }
        }
        if (j0 + 4 > D) m &= (1u << (D - j0)) - 1u;
      }
      mks |= (unsigned long long)m << (4 * k);
    }
    // donor genes of the masked slots, Eq. (1) and the clip
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kSpanVmax; ++k) {
      if (k * G >= D4) break;                    // no lane holds slot k or later
      const unsigned m = (unsigned)(mks >> (4 * k)) & 0xFu;
      if (m) {
        const int q = gl + k * G;
        const float4 a1 = ld_ro(d1 + q), a2 = ld_ro(d2 + q), a3 = ld_ro(d3 + q);
        if (m & 1u) x[k].x = clip_box(mutate(a1.x, a2.x, a3.x, F), lo, hi);
        if (m & 2u) x[k].y = clip_box(mutate(a1.y, a2.y, a3.y, F), lo, hi);
        if (m & 4u) x[k].z = clip_box(mutate(a1.z, a2.z, a3.z, F), lo, hi);
        if (m & 8u) x[k].w = clip_box(mutate(a1.w, a2.w, a3.w, F), lo, hi);
        if (XO == kBin) cnt += __popc(m);
      }
    }

    // fitness partials: slot k goes to accumulator set k mod R (virtual lane gl + G (k mod R))
    Acc s[R];
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = Acc{0.0f, 0.0f, 0.0f};
    if constexpr (OBJ == kRosenbrock) {
#pragma unroll
      for (int k = 0; k < kSpanVmax; ++k) {
        if (k * G >= D4) break;                    // no lane holds slot k or later
        float nb = __shfl_down_sync(0xFFFFFFFFu, x[k].x, 1, G);
        const float next0 = __shfl_sync(0xFFFFFFFFu, (k + 1 < kSpanVmax) ? x[k + 1].x : 0.0f, 0, G);
        if (gl == G - 1) nb = next0;               // group lane 0, next slot
        const int q = gl + k * G;
        if (active && q < D4) {
          Acc& a = s[k % R];
          const int j0 = 4 * q;
          if (j0 + 4 < D) {
            accum_pair(a, x[k].x, x[k].y);
            accum_pair(a, x[k].y, x[k].z);
            accum_pair(a, x[k].z, x[k].w);
            accum_pair(a, x[k].w, nb);
          } else {
            if (j0 + 1 < D) accum_pair(a, x[k].x, x[k].y);
            if (j0 + 2 < D) accum_pair(a, x[k].y, x[k].z);
            if (j0 + 3 < D) accum_pair(a, x[k].z, x[k].w);
          }
        }
      }
    } else {
      if (active) {
#pragma unroll
        for (int k = 0; k < kSpanVmax; ++k) {
          if (k * G >= D4) break;                    // no lane holds slot k or later
          const int q = gl + k * G;
          if (q < D4) {
            Acc& a = s[k % R];
            const int j0 = 4 * q;
            if (j0 + 4 <= D) {
              accum_gene<OBJ>(a, x[k].x, j0, p);
              accum_gene<OBJ>(a, x[k].y, j0 + 1, p);
              accum_gene<OBJ>(a, x[k].z, j0 + 2, p);
              accum_gene<OBJ>(a, x[k].w, j0 + 3, p);
            } else {
              accum_gene<OBJ>(a, x[k].x, j0, p);
              if (j0 + 1 < D) accum_gene<OBJ>(a, x[k].y, j0 + 1, p);
              if (j0 + 2 < D) accum_gene<OBJ>(a, x[k].z, j0 + 2, p);
            }
          }
        }
      }
    }
    // butterfly over the 32 virtual lanes: strides >= G inside the lane, the rest by shuffles
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= G) {
        const int b = o / G;
#pragma unroll
        for (int t = 0; t < R; ++t)
          if (!(t & b)) {
            s[t].a += s[t | b].a;
            if (NS > 1) s[t].b += s[t | b].b;
            if (NS > 2) s[t].c += s[t | b].c;
          }
      } else {
        s[0].a += __shfl_xor_sync(0xFFFFFFFFu, s[0].a, o, G);
        if (NS > 1) s[0].b += __shfl_xor_sync(0xFFFFFFFFu, s[0].b, o, G);
        if (NS > 2) s[0].c += __shfl_xor_sync(0xFFFFFFFFu, s[0].c, o, G);
      }
    }
    if (XO == kBin) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o, G);
    }

    // decision by the group leader
    int acc = 0;
    if (active && gl == 0) {
      float f = finalize_fitness<OBJ>(s[0], p);
      if (f != f) f = __int_as_float(0x7F800000);
      if (eval_only) {
        p.fit[i] = f;
        const unsigned long long key = best_key_of(f, i);
        kmin = key < kmin ? key : kmin;
      } else {
        acc = (f < pl.fit_i) ? 1 : 0;
        slot_out[i] = (uint8_t)(acc ? 1 - si : si);
        const int Lrow = (XO == kBin) ? cnt : pl.L;
        masked_sum += (unsigned long long)Lrow;
        accepts += (unsigned)acc;
        if (acc) {
          p.fit[i] = f;
          const unsigned long long key = best_key_of(f, i);
          kmin = key < kmin ? key : kmin;
        }
        if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
        if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
        if (p.dbg_draws) {
          int* o = p.dbg_draws + 5 * (size_t)i;
          o[0] = pl.r1; o[1] = pl.r2; o[2] = pl.r3; o[3] = pl.jrand; o[4] = Lrow;
        }
      }
    }
    acc = __shfl_sync(0xFFFFFFFFu, acc, gi * G);   // the group leader's decision
    if (active && !eval_only) {
      if (acc) {
        float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * pitch);
#pragma unroll
        for (int k = 0; k < kSpanVmax; ++k) {
          if (k * G >= D4) break;                    // no lane holds slot k or later
          const int q = gl + k * G;
          if (q < D4) st_stream(out + q, x[k]);
        }
      }
      if (p.dbg_trial) {
        float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * pitch);
#pragma unroll
        for (int k = 0; k < kSpanVmax; ++k) {
          if (k * G >= D4) break;                    // no lane holds slot k or later
          const int q = gl + k * G;
          if (q < D4) o[q] = x[k];
        }
      }
    }
  }

  // the span's counters go to the instance state once
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ko = __shfl_xor_sync(0xFFFFFFFFu, kmin, o);
    kmin = ko < kmin ? ko : kmin;
    masked_sum += __shfl_xor_sync(0xFFFFFFFFu, masked_sum, o);
    accepts += __shfl_xor_sync(0xFFFFFFFFu, accepts, o);
  }
  if (lane == 0) {
    if (kmin != ~0ull) atomicMin(&p.st->best_key, kmin);
    if (!eval_only) {
      if (accepts) atomicAdd(&p.st->accepts, (unsigned long long)accepts);
      atomicAdd(&p.st->masked, masked_sum);
    }
  }
}

template <int OBJ, int XO>
__device__ __forceinline__ void span_rows_g(int G, const BatchInst* Ip, int row0, int rows, const RowPlan32* spl,
                                            int eval_only) {
  switch (G) {
    case 4: span_rows<OBJ, XO, 4>(Ip, row0, rows, spl, eval_only); break;
    case 8: span_rows<OBJ, XO, 8>(Ip, row0, rows, spl, eval_only); break;
    case 16: span_rows<OBJ, XO, 16>(Ip, row0, rows, spl, eval_only); break;
    default: span_rows<OBJ, XO, 32>(Ip, row0, rows, spl, eval_only); break;
  }
}

// Spans of crossover XO. ctr[0]: next span to take; ctr[1]: warps finished.
// The last warp to finish resets both, so every launch starts from zero.
template <int XO>
__global__ void __launch_bounds__(kSpanThreads, 2)
batch_span_kernel(const BatchInst* __restrict__ insts, const BatchSpan* __restrict__ spans, int nspans,
                  const RowPlan32* __restrict__ plans, unsigned* ctr, int eval_only) {
  __shared__ __align__(16) RowPlan32 s_plan[kSpanThreads / 32][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  RowPlan32* spl = s_plan[warp];
  for (;;) {
    unsigned idx = 0u;
    if (lane == 0) idx = atomicAdd(&ctr[0], 1u);
    idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
    if (idx >= (unsigned)nspans) break;
    const BatchSpan sp = spans[idx];
    if (!eval_only) {
      if (lane < sp.rows) {
        const uint4* src = reinterpret_cast<const uint4*>(plans + sp.plan0 + lane);
        uint4* dst = reinterpret_cast<uint4*>(spl + lane);
        const uint4 w0 = __ldcs(src), w1 = __ldcs(src + 1);
        dst[0] = w0;
        dst[1] = w1;
      }
      __syncwarp();
    }
    const BatchInst* Ip = insts + sp.inst;
    const int obj = Ip->obj, G = Ip->group;          // uniform over the warp
    switch (obj) {
      case kSphere: span_rows_g<kSphere, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
      case kRastrigin: span_rows_g<kRastrigin, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
      case kAckley: span_rows_g<kAckley, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
      case kRosenbrock: span_rows_g<kRosenbrock, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
      case kGriewank: span_rows_g<kGriewank, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
      default: span_rows_g<kElliptic, XO>(G, Ip, sp.row0, sp.rows, spl, eval_only); break;
    }
    __syncwarp();                                     // plans read before the next span overwrites them
  }
  if (lane == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctr[1], 1u);
    if (done == gridDim.x * (kSpanThreads / 32) - 1u) {
      ctr[0] = 0u;
      ctr[1] = 0u;
      __threadfence();
    }
  }
}

template <int XO>
cudaError_t launch_batch_span_xo(const BatchInst* insts, const BatchSpan* spans, int nspans, const RowPlan32* plans,
                                 unsigned* ctr, int eval_only, int grid, cudaStream_t s) {
  batch_span_kernel<XO><<<grid, kSpanThreads, 0, s>>>(insts, spans, nspans, plans, ctr, eval_only);
  return cudaGetLastError();
}

}  // namespace de
