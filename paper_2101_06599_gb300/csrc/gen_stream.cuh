// gen_stream.cuh — the streaming generation kernel: one warp per row, the
// row processed in chunks of 32 x kStreamU float4 slots, nothing of it kept.
//
// Pass 1 computes the trial chunk by chunk (parent loads first, then the
// crossover masks, then the three donor float4s of every slot holding a
// masked gene, all issued before any is used: Alg. 2 order, mutation of
// masked genes only) and accumulates the objective's partial sums in
// registers. The warp reduces them, selects (strict '<', NaN as +inf), and
// only a row that wins recomputes its trial in pass 2 and stores it to the
// other slot buffer; donors are never written during a generation, so pass 2
// reproduces pass 1 exactly. Binomial masks (one Philox block per slot) are
// kept in shared memory by pass 1, one byte per slot of the warp's row, so
// pass 2 reads them instead of drawing them again. This suits the binomial crossover at large D:
// nearly every donor gene is needed (m ~ Cr), so the row-per-CTA kernel's
// registers hold four rows' worth of loads per row and few rows fit per SM,
// while here 16 rows per SM stream with all their loads in flight.
#pragma once
#include "draws.cuh"
#include "objectives.cuh"

namespace de {

constexpr int kStreamWarps = 8;    // rows per CTA
constexpr int kStreamU = 2;        // float4 slots per lane per chunk

struct StreamRow {
  const float4* x;                 // parent row
  const float4* d1;
  const float4* d2;
  const float4* d3;
  int jrand, L, i;
  uint32_t g;
};

// The trial slots q = q0 + lane + 32 u of row r; m[u] gets the mask bits.
// Binomial: the masks are drawn and written to mc[q] (pass 1, kCached false)
// or read back from it (pass 2).
template <int XO, bool kCached, int kRepair>
__device__ __forceinline__ void stream_trial_chunk(const GenParams& p, const StreamRow& r, int q0, int lane,
                                                   float4 (&v)[kStreamU], unsigned (&m)[kStreamU], uint8_t* mc) {
#pragma unroll
  for (int u = 0; u < kStreamU; ++u) {
    const int q = q0 + lane + 32 * u;
    v[u] = (q < p.D4) ? ld_stream(r.x + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
#pragma unroll
  for (int u = 0; u < kStreamU; ++u) {
    const int q = q0 + lane + 32 * u;
    unsigned mm = 0u;
    if (q < p.D4) {
      const int j0 = 4 * q;
      if constexpr (XO == kBin && kCached) {
        mm = mc[q];
      } else if constexpr (XO == kBin) {
        mm = bin_mask(p, philox_block_rk(p.rk, kStreamBin, p.inst, r.g, (uint32_t)r.i, (uint32_t)q), q, r.jrand);
      } else {
        int dd = j0 - r.jrand;
        if (dd < 0) dd += p.D;                      // (j0 - j_rand) mod D
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int de = dd + e;
          if (de >= p.D) de -= p.D;
          mm |= (de < r.L) ? (1u << e) : 0u;
        }
      }
      mm &= (1u << min(4, p.D - j0)) - 1u;          // padding genes never cross
      if constexpr (XO == kBin && !kCached) mc[q] = (uint8_t)mm;
    }
    m[u] = mm;
  }
  float4 a1[kStreamU], a2[kStreamU], a3[kStreamU];
#pragma unroll
  for (int u = 0; u < kStreamU; ++u) {
    const int q = q0 + lane + 32 * u;
    if (m[u]) {
      a1[u] = ld_ro(r.d1 + q);
      a2[u] = ld_ro(r.d2 + q);
      a3[u] = ld_ro(r.d3 + q);
    }
  }
#pragma unroll
  for (int u = 0; u < kStreamU; ++u) {
    if (m[u]) mutate_slot<kRepair>(v[u], a1[u], a2[u], a3[u], m[u], p);
  }
}

// Pass 1 of one row: the trial chunk by chunk, its objective (even and odd
// slots of a chunk into two independent partial sums: shorter dependency
// chains) reduced over the warp; every lane returns the value (NaN as +inf).
// cnt gets the binomial mask's popcount. Writes the trial to p.dbg_trial when set.
template <int XO, int OBJ, int kRepair>
__device__ __forceinline__ float stream_row_value(const GenParams& p, const StreamRow& r, int lane, int& cnt,
                                                  uint8_t* mc) {
  Acc s{0.0f, 0.0f, 0.0f}, s2{0.0f, 0.0f, 0.0f};
  cnt = 0;
  float carry = 0.0f;                              // Rosenbrock: last gene of the previous chunk
  for (int q0 = 0; q0 < p.D4; q0 += 32 * kStreamU) {
    float4 v[kStreamU];
    unsigned m[kStreamU];
    stream_trial_chunk<XO, false, kRepair>(p, r, q0, lane, v, m, mc);
    if (p.dbg_trial) {
      float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)r.i * p.pitch);
#pragma unroll
      for (int u = 0; u < kStreamU; ++u) {
        const int q = q0 + lane + 32 * u;
        if (q < p.D4) o[q] = v[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kStreamU; ++u) {
      if constexpr (XO == kBin) cnt += __popc(m[u]);
      const int q = q0 + lane + 32 * u;
      const int j0 = 4 * q;
      Acc& su = (u & 1) ? s2 : s;
      if constexpr (OBJ == kRosenbrock) {
        float nb = __shfl_down_sync(0xFFFFFFFFu, v[u].x, 1);
        const float first_next = (u + 1 < kStreamU) ? __shfl_sync(0xFFFFFFFFu, v[(u + 1) % kStreamU].x, 0) : 0.0f;
        if (lane == 31) nb = first_next;
        if (u == 0 && lane == 0 && q0 > 0) accum_pair(su, carry, v[0].x);   // the pair across chunks
        if (q < p.D4) {
          if (j0 + 1 < p.D) accum_pair(su, v[u].x, v[u].y);
          if (j0 + 2 < p.D) accum_pair(su, v[u].y, v[u].z);
          if (j0 + 3 < p.D) accum_pair(su, v[u].z, v[u].w);
          if (j0 + 4 < p.D && !(lane == 31 && u + 1 == kStreamU)) accum_pair(su, v[u].w, nb);
        }
      } else {
        if (j0 + 4 <= p.D) {                       // a full slot: the common case
          accum_gene<OBJ>(su, v[u].x, j0, p);
          accum_gene<OBJ>(su, v[u].y, j0 + 1, p);
          accum_gene<OBJ>(su, v[u].z, j0 + 2, p);
          accum_gene<OBJ>(su, v[u].w, j0 + 3, p);
        } else if (q < p.D4) {
          accum_gene<OBJ>(su, v[u].x, j0, p);
          if (j0 + 1 < p.D) accum_gene<OBJ>(su, v[u].y, j0 + 1, p);
          if (j0 + 2 < p.D) accum_gene<OBJ>(su, v[u].z, j0 + 2, p);
        }
      }
    }
    if constexpr (OBJ == kRosenbrock) carry = __shfl_sync(0xFFFFFFFFu, v[kStreamU - 1].w, 31);
  }
  s.a += s2.a;
  s.b += s2.b;
  s.c += s2.c;
  constexpr int NS = ObjTraits<OBJ>::kSums;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.a += __shfl_xor_sync(0xFFFFFFFFu, s.a, o);
    if (NS > 1) s.b += __shfl_xor_sync(0xFFFFFFFFu, s.b, o);
    if (NS > 2) s.c += __shfl_xor_sync(0xFFFFFFFFu, s.c, o);
    if (XO == kBin) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  }
  float f = finalize_fitness<OBJ>(s, p);
  if (f != f) f = __int_as_float(0x7F800000);     // NaN counts as +inf
  return f;
}

// Pass 2 of a winning row: its trial again, chunk by chunk, stored to `out`.
template <int XO, int kRepair>
__device__ __forceinline__ void stream_row_store(const GenParams& p, const StreamRow& r, int lane, float4* out,
                                                 uint8_t* mc) {
  for (int q0 = 0; q0 < p.D4; q0 += 32 * kStreamU) {
    float4 v[kStreamU];
    unsigned m[kStreamU];
    stream_trial_chunk<XO, true, kRepair>(p, r, q0, lane, v, m, mc);
#pragma unroll
    for (int u = 0; u < kStreamU; ++u) {
      const int q = q0 + lane + 32 * u;
      if (q < p.D4) st_stream(out + q, v[u]);
    }
  }
}

template <int XO, int OBJ>
__global__ void __launch_bounds__(kStreamWarps * 32, 4) gen_stream_kernel(const __grid_constant__ GenParams p) {
  __shared__ unsigned long long s_key[kStreamWarps];
  __shared__ int s_cnt[kStreamWarps];
  __shared__ int s_acc[kStreamWarps];
  extern __shared__ uint8_t s_masks[];             // binomial: D4 mask bytes per warp
  griddep_wait();                                  // the previous generation has closed
  griddep_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* mc = (XO == kBin) ? s_masks + (size_t)warp * p.D4 : nullptr;
  const int i = blockIdx.x * kStreamWarps + warp;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  unsigned long long key = ~0ull;
  int Lrow = 0, acc = 0;
  if (i < p.N) {                                     // warp-uniform
    const int si = slot_in[i];
    const float fi = p.fit[i];                       // needed at the selection; loaded off the row's chain
    StreamRow r;
    r.x = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)i * p.pitch);
    r.i = i;
    r.g = g;
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
    r.jrand = __shfl_sync(0xFFFFFFFFu, d.jrand, 0);
    r.L = __shfl_sync(0xFFFFFFFFu, d.L, 0);
    r.d1 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd1, 0));
    r.d2 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd2, 0));
    r.d3 = reinterpret_cast<const float4*>(__shfl_sync(0xFFFFFFFFu, pd3, 0));

    int cnt = 0;
    // the repair mode is uniform across the launch: one copy of the row code each
    const float f = p.repair ? stream_row_value<XO, OBJ, 1>(p, r, lane, cnt, mc)
                             : stream_row_value<XO, OBJ, 0>(p, r, lane, cnt, mc);
    acc = (f < fi) ? 1 : 0;
    __syncwarp();                                    // every lane has read fit[i] before lane 0 writes it
    Lrow = (XO == kBin) ? cnt : r.L;
    if (lane == 0) {
      slot_out[i] = (uint8_t)(acc ? 1 - si : si);
      if (acc) p.fit[i] = f;
      if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
      if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
      if (p.dbg_draws) {
        int* o = p.dbg_draws + 5 * (size_t)i;
        o[0] = d.r1; o[1] = d.r2; o[2] = d.r3; o[3] = d.jrand; o[4] = Lrow;
      }
    }
    if (acc) {
      key = best_key_of(f, i);
      // pass 2: the winning trial again, into the other slot buffer
      float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
      __syncwarp();                                  // every lane's mask bytes are written
      if (p.repair) stream_row_store<XO, 1>(p, r, lane, out, mc);
      else stream_row_store<XO, 0>(p, r, lane, out, mc);
    }
  }
  if (lane == 0) {
    s_key[warp] = key;
    s_cnt[warp] = Lrow;
    s_acc[warp] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long k = ~0ull, masked = 0;
    unsigned long long accepts = 0;
    for (int w = 0; w < kStreamWarps; ++w) {
      k = (s_key[w] < k) ? s_key[w] : k;
      masked += (unsigned long long)s_cnt[w];
      accepts += (unsigned long long)s_acc[w];
    }
    if (accepts) {
      atomicMin(&p.st->best_key, k);
      atomicAdd(&p.st->accepts, accepts);
    }
    atomicAdd(&p.st->masked, masked);
    // the last CTA closes the generation
    __threadfence();
    const unsigned prev = atomicAdd(&p.st->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const unsigned long long bk = atomicAdd(&p.st->best_key, 0ULL);
      const float bf = from_ordered_bits((uint32_t)(bk >> 32));
      if (bf < p.st->best_f) {
        p.st->best_f = bf;
        p.st->best_gen = gen + 1;
      }
      p.st->gen = gen + 1;
      p.st->base_row = (int)(uint32_t)(bk & 0xFFFFFFFFull);
      p.st->done = 0u;
    }
  }
}

// Dynamic shared memory of a launch: the binomial mask bytes, kStreamWarps x
// D4 (at most 64 KB, D <= 32768; prepare_stream_obj allows that much).
constexpr int kStreamMaskSmemMax = kStreamWarps * 8192;

template <int XO, int OBJ>
cudaError_t prepare_stream_obj() {
  if (XO != kBin) return cudaSuccess;
  return cudaFuncSetAttribute(gen_stream_kernel<XO, OBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kStreamMaskSmemMax);
}

template <int XO, int OBJ>
cudaError_t launch_stream_obj(const GenParams& p, cudaStream_t s) {
  const unsigned grid = (unsigned)((p.N + kStreamWarps - 1) / kStreamWarps);
  const size_t smem = (XO == kBin) ? (size_t)kStreamWarps * (size_t)p.D4 : 0;
  return launch_pdl(gen_stream_kernel<XO, OBJ>, dim3(grid), dim3(kStreamWarps * 32), smem, s, p);
}

template <int XO>
cudaError_t prepare_stream_xo(int obj) {
  switch (obj) {
    case kSphere: return prepare_stream_obj<XO, kSphere>();
    case kRastrigin: return prepare_stream_obj<XO, kRastrigin>();
    case kAckley: return prepare_stream_obj<XO, kAckley>();
    case kRosenbrock: return prepare_stream_obj<XO, kRosenbrock>();
    case kGriewank: return prepare_stream_obj<XO, kGriewank>();
    case kElliptic: return prepare_stream_obj<XO, kElliptic>();
    default: return cudaErrorInvalidValue;
  }
}

template <int XO>
cudaError_t launch_stream_xo(int obj, const GenParams& p, cudaStream_t s) {
  switch (obj) {
    case kSphere: return launch_stream_obj<XO, kSphere>(p, s);
    case kRastrigin: return launch_stream_obj<XO, kRastrigin>(p, s);
    case kAckley: return launch_stream_obj<XO, kAckley>(p, s);
    case kRosenbrock: return launch_stream_obj<XO, kRosenbrock>(p, s);
    case kGriewank: return launch_stream_obj<XO, kGriewank>(p, s);
    case kElliptic: return launch_stream_obj<XO, kElliptic>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace de
