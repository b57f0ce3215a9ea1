// gen_kernel.cuh — the fused DE/rand/1 generation kernel (Alg. 2, one loop
// iteration, for every row at once) and the row-fitness block reduction it
// shares with the evaluation kernel.
//
// One CTA owns one row i. Its T threads hold the row in registers as V
// float4 slots each (slot q = t + k T, genes 4q .. 4q+3), so the parent row
// is read from HBM exactly once with coalesced 128-bit loads. Per row:
//   1. every thread issues its parent loads; meanwhile thread 0 draws r1,
//      r2, r3, j_rand and publishes the donor rows, and the first thread of
//      the second warp draws L for exp / NEC (both at once);
//   2. each thread computes the crossover mask of its genes in registers
//      (binomial: one Philox block per slot; exp / NEC: the circular test
//      ((j - j_rand) mod D) < L) and, only for slots holding a masked gene,
//      loads the three donor float4s and applies Eq. (1) plus clipping —
//      the mutation is never computed for genes the mask discards
//      (Section 2, after Eq. 1);
//   3. FP32 partial sums of the objective, warp shuffles, one smem pass;
//   4. thread 0 compares with fit[i] (strict '<', NaN as +inf), updates the
//      fitness, slot bit, counters and best key;
//   5. if accepted, the row (still in registers) is stored to the other
//      slot buffer; the last CTA to finish closes the generation (best
//      generation, generation counter) — no CTA ever waits on another.
#pragma once
#include "draws.cuh"
#include "objectives.cuh"

namespace de {

struct RowShared {
  const float4* d1;
  const float4* d2;
  const float4* d3;
  int r1, r2, r3, jrand, L;
  int accept;
};

__device__ __forceinline__ void warp_reduce(Acc& s, int& cnt, int ns) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.a += __shfl_xor_sync(0xFFFFFFFFu, s.a, o);
    if (ns > 1) s.b += __shfl_xor_sync(0xFFFFFFFFu, s.b, o);
    if (ns > 2) s.c += __shfl_xor_sync(0xFFFFFFFFu, s.c, o);
    cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  }
}

// Row fitness of the values in x (this thread's slots). `cnt` is summed
// alongside. The result is valid in thread 0 only. Uses two barriers
// (three for Rosenbrock). blockDim.x must be a multiple of 32.
template <int OBJ, int V>
__device__ __forceinline__ float block_row_fitness(const float4 (&x)[V], int& cnt, const GenParams& p,
                                                   float (*s_first)[32], float (*red)[32]) {
  const int t = threadIdx.x, T = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = T >> 5;
  Acc s{0.0f, 0.0f, 0.0f};
  if constexpr (OBJ == kRosenbrock) {
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < V; ++k) s_first[k][warp] = x[k].x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float nb = __shfl_down_sync(0xFFFFFFFFu, x[k].x, 1);
      if (lane == 31) nb = (warp + 1 < nwarps) ? s_first[k][warp + 1] : (k + 1 < V ? s_first[k + 1][0] : 0.0f);
      const int q = t + k * T;
      if (q < p.D4) {
        const int j0 = 4 * q;
        if (j0 + 1 < p.D) accum_pair(s, x[k].x, x[k].y);
        if (j0 + 2 < p.D) accum_pair(s, x[k].y, x[k].z);
        if (j0 + 3 < p.D) accum_pair(s, x[k].z, x[k].w);
        if (j0 + 4 < p.D) accum_pair(s, x[k].w, nb);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int q = t + k * T;
      if (q < p.D4) {
        const int j0 = 4 * q;
        accum_gene<OBJ>(s, x[k].x, j0, p);
        if (j0 + 1 < p.D) accum_gene<OBJ>(s, x[k].y, j0 + 1, p);
        if (j0 + 2 < p.D) accum_gene<OBJ>(s, x[k].z, j0 + 2, p);
        if (j0 + 3 < p.D) accum_gene<OBJ>(s, x[k].w, j0 + 3, p);
      }
    }
  }
  constexpr int NS = ObjTraits<OBJ>::kSums;
  warp_reduce(s, cnt, NS);
  if (lane == 0) {
    red[0][warp] = s.a;
    red[1][warp] = s.b;
    red[2][warp] = s.c;
    red[3][warp] = __int_as_float(cnt);
  }
  __syncthreads();
  float f = 0.0f;
  if (warp == 0) {
    Acc r{0.0f, 0.0f, 0.0f};
    int c = 0;
    if (lane < nwarps) {
      r.a = red[0][lane];
      r.b = red[1][lane];
      r.c = red[2][lane];
      c = __float_as_int(red[3][lane]);
    }
    warp_reduce(r, c, NS);
    cnt = c;
    f = finalize_fitness<OBJ>(r, p);
    if (f != f) f = __int_as_float(0x7F800000);   // NaN counts as +inf
  }
  return f;
}

template <int XO, int OBJ, int V>
__global__ void __launch_bounds__(kMaxThreads) gen_kernel(const __grid_constant__ GenParams p) {
  __shared__ RowShared sh;
  __shared__ float red[4][32];
  __shared__ float s_first[(OBJ == kRosenbrock) ? V : 1][32];

  griddep_wait();                                  // the previous generation has closed
  griddep_launch_dependents();
  const int i = blockIdx.x;
  const int t = threadIdx.x, T = blockDim.x;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  const int si = slot_in[i];
  const float4* xrow = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)i * p.pitch);
  // the parent's fitness is only needed at the selection: load it now, off
  // the generation's chain of dependent steps
  const float fi = (t == 0) ? p.fit[i] : 0.0f;

  // 1. parent row -> registers (all loads in flight before anything waits)
  float4 x[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int q = t + k * T;
    x[k] = (q < p.D4) ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }

  // draws, once per row: the donors on thread 0 and, at the same time, the
  // segment length on the first thread of the second warp (thread 0 as well
  // when the CTA is a single warp)
  const int tlen = (T >= 64) ? 32 : 0;
  if (t == 0) {
    RowDraws d;
    draw_donors(p, g, i, d);
    sh.r1 = d.r1; sh.r2 = d.r2; sh.r3 = d.r3; sh.jrand = d.jrand;
    sh.d1 = reinterpret_cast<const float4*>((slot_in[d.r1] ? p.pop1 : p.pop0) + (size_t)d.r1 * p.pitch);
    sh.d2 = reinterpret_cast<const float4*>((slot_in[d.r2] ? p.pop1 : p.pop0) + (size_t)d.r2 * p.pitch);
    sh.d3 = reinterpret_cast<const float4*>((slot_in[d.r3] ? p.pop1 : p.pop0) + (size_t)d.r3 * p.pitch);
  }
  if (t == tlen) {
    int L = 0;
    if constexpr (XO == kNec) L = nec_length(p, g, i);
    else if constexpr (XO == kExp) L = exp_walk_length(p, g, i);
    sh.L = L;
  }
  __syncthreads();

  // 2. crossover mask + mutation of masked genes only
  const int jrand = sh.jrand, L = sh.L;
  const float4* d1 = sh.d1;
  const float4* d2 = sh.d2;
  const float4* d3 = sh.d3;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int q = t + k * T;
    if (q < p.D4) {
      const int j0 = 4 * q;
      unsigned m = 0u;
      if constexpr (XO == kBin) {
        m = bin_mask(p, philox_block_rk(p.rk, kStreamBin, p.inst, g, (uint32_t)i, (uint32_t)q), q, jrand);
      } else {
        int dd = j0 - jrand;
        if (dd < 0) dd += p.D;                      // (j0 - j_rand) mod D
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int de = dd + e;
          if (de >= p.D) de -= p.D;
          m |= (de < L) ? (1u << e) : 0u;
        }
      }
      const int valid = min(4, p.D - j0);
      m &= (1u << valid) - 1u;                      // padding genes never cross
      if (m) {
        const float4 a1 = ld_ro(d1 + q), a2 = ld_ro(d2 + q), a3 = ld_ro(d3 + q);
        mutate_slot(x[k], a1, a2, a3, m, p);
      }
      if constexpr (XO == kBin) cnt += __popc(m);
    }
  }

  // 3. fitness of the trial
  const float f = block_row_fitness<OBJ, V>(x, cnt, p, s_first, red);

  // 4. selection (thread 0)
  if (t == 0) {
    const int acc = (f < fi) ? 1 : 0;
    sh.accept = acc;
    slot_out[i] = (uint8_t)(acc ? 1 - si : si);
    const int Lrow = (XO == kBin) ? cnt : L;
    if (acc) {
      p.fit[i] = f;
      atomicMin(&p.st->best_key, best_key_of(f, i));
      atomicAdd(&p.st->accepts, 1ULL);
    }
    atomicAdd(&p.st->masked, (unsigned long long)Lrow);
    if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
    if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
    if (p.dbg_draws) {
      int* o = p.dbg_draws + 5 * (size_t)i;
      o[0] = sh.r1; o[1] = sh.r2; o[2] = sh.r3; o[3] = sh.jrand; o[4] = Lrow;
    }
  }
  __syncthreads();

  // 5. accepted rows go to the other slot buffer
  if (sh.accept) {
    float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int q = t + k * T;
      if (q < p.D4) st_stream(out + q, x[k]);
    }
  }
  if (p.dbg_trial) {
    float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * p.pitch);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int q = t + k * T;
      if (q < p.D4) o[q] = x[k];
    }
  }

  // the last CTA closes the generation
  if (t == 0) {
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

template <int XO, int OBJ>
cudaError_t launch_gen_obj(int vidx, const GenParams& p, int block, cudaStream_t s) {
  const dim3 grid((unsigned)p.N), blk((unsigned)block);
  switch (vidx) {
    case 0: return launch_pdl(gen_kernel<XO, OBJ, 1>, grid, blk, 0, s, p);
    case 1: return launch_pdl(gen_kernel<XO, OBJ, 2>, grid, blk, 0, s, p);
    case 2: return launch_pdl(gen_kernel<XO, OBJ, 4>, grid, blk, 0, s, p);
    case 3: return launch_pdl(gen_kernel<XO, OBJ, 8>, grid, blk, 0, s, p);
    case 4: return launch_pdl(gen_kernel<XO, OBJ, 16>, grid, blk, 0, s, p);
    default: return cudaErrorInvalidValue;
  }
}

template <int XO>
cudaError_t launch_gen_xo(int obj, int vidx, const GenParams& p, int block, cudaStream_t s) {
  switch (obj) {
    case kSphere: return launch_gen_obj<XO, kSphere>(vidx, p, block, s);
    case kRastrigin: return launch_gen_obj<XO, kRastrigin>(vidx, p, block, s);
    case kAckley: return launch_gen_obj<XO, kAckley>(vidx, p, block, s);
    case kRosenbrock: return launch_gen_obj<XO, kRosenbrock>(vidx, p, block, s);
    case kGriewank: return launch_gen_obj<XO, kGriewank>(vidx, p, block, s);
    case kElliptic: return launch_gen_obj<XO, kElliptic>(vidx, p, block, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace de
