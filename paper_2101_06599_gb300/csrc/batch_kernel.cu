// batch_kernel.cu — one generation of many independent DE instances (each
// with its own N, D, objective, crossover, Cr, F, box and Philox instance
// field) in a single launch.
//
// The host cuts every instance into tiles of R = 256 / G rows, G threads per
// row (G a power of two, 4..256, per instance: the tile shape). The grid
// walks the tile list (longest-processing-time order) with a grid stride.
// Inside a tile each row is handled by its group of G threads exactly as the
// row-per-CTA kernel handles a row: parent row in registers (up to 16 float4
// per thread), draws by the group leader (NEC thresholds staged in shared
// memory), crossover mask and mutation of the masked genes, FP32 fitness
// reduced over the group, strict selection, accepted rows stored to the
// other slot buffer. Counters are summed per tile; the last tile of an
// instance to finish closes that instance's generation, so instances never
// wait for each other. With eval_only the same kernel evaluates the parents
// (the initial evaluation), so stored and trial fitness share one reduction
// order.
#include "draws.cuh"
#include "gen_kernel.cuh"
#include "internal.h"
#include "objectives.cuh"

namespace de {

constexpr int kBatchThreads = 256;
constexpr int kBatchVmax = 16;
constexpr int kBatchTableCap = 2048;

__device__ __forceinline__ void accum_gene_rt(int obj, Acc& s, float x, int j, const GenParams& p) {
  switch (obj) {
    case kSphere: accum_gene<kSphere>(s, x, j, p); break;
    case kRastrigin: accum_gene<kRastrigin>(s, x, j, p); break;
    case kAckley: accum_gene<kAckley>(s, x, j, p); break;
    case kGriewank: accum_gene<kGriewank>(s, x, j, p); break;
    default: accum_gene<kElliptic>(s, x, j, p); break;
  }
}

__device__ __forceinline__ float finalize_rt(int obj, const Acc& s, const GenParams& p) {
  switch (obj) {
    case kAckley: return finalize_fitness<kAckley>(s, p);
    case kGriewank: return finalize_fitness<kGriewank>(s, p);
    default: return s.a;
  }
}

struct BatchRowShared {
  const float4* d1;
  const float4* d2;
  const float4* d3;
  int r1, r2, r3, jrand, L, si, accept;
};

__global__ void __launch_bounds__(kBatchThreads, 2)
batch_gen_kernel(const BatchInst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                 int eval_only) {
  __shared__ BatchInst sI;
  __shared__ uint32_t s_tab[kBatchTableCap];
  __shared__ BatchRowShared s_row[kBatchThreads / 4];
  __shared__ float s_first[kBatchVmax][kBatchThreads / 32];
  __shared__ float s_red[4][kBatchThreads / 32];
  __shared__ unsigned long long s_acc, s_msk;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const BatchTile tl = tiles[tile];
    if (t == 0) {
      sI = insts[tl.inst];
      s_acc = 0ull;
      s_msk = 0ull;
    }
    __syncthreads();
    const GenParams& p = sI.g;
    const int obj = sI.obj, xo = sI.xo, G = sI.group;
    const bool tab_smem = (xo == kNec) && p.nT <= kBatchTableCap;
    if (tab_smem)
      for (int k = t; k < p.nT; k += kBatchThreads) s_tab[k] = p.nec_tm1[k];

    const long long gen = p.st->gen;
    const uint32_t g = (uint32_t)gen;
    const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
    uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
    const int gi = t / G, gl = t - gi * G;          // row within the tile, lane within the row's group
    const int i = tl.row0 + gi;
    const bool active = i < p.N;

    // parent row -> registers
    float4 x[kBatchVmax];
    int si = 0;
    if (active) si = slot_in[i];
    const float4* xrow = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)(active ? i : 0) * p.pitch);
#pragma unroll
    for (int k = 0; k < kBatchVmax; ++k) {
      const int q = gl + k * G;
      x[k] = (active && q < p.D4) ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();                                 // threshold table staged

    if (active && gl == 0 && !eval_only) {
      RowDraws d;
      draw_donors(p, g, i, d);
      int L = 0;
      if (xo == kNec) {
        if (p.cr_mode == kCrZero) L = 1;
        else if (p.cr_mode == kCrOne) L = p.D;
        else {
          const uint32_t w = philox_block(p.key, kStreamLen, p.inst, g, (uint32_t)i, 0u).x;
          if (w == 0u) {
            L = p.D;
          } else {
            int lo = 0, hi = min(p.D - 1, p.nT);
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              const uint32_t tv = tab_smem ? s_tab[mid - 1] : __ldg(p.nec_tm1 + (mid - 1));
              if (w <= tv) lo = mid; else hi = mid - 1;
            }
            L = 1 + lo;
          }
        }
      } else if (xo == kExp) {
        L = exp_walk_length(p, g, i);
      }
      BatchRowShared& r = s_row[gi];
      r.r1 = d.r1; r.r2 = d.r2; r.r3 = d.r3; r.jrand = d.jrand; r.L = L; r.si = si;
      r.d1 = reinterpret_cast<const float4*>((slot_in[d.r1] ? p.pop1 : p.pop0) + (size_t)d.r1 * p.pitch);
      r.d2 = reinterpret_cast<const float4*>((slot_in[d.r2] ? p.pop1 : p.pop0) + (size_t)d.r2 * p.pitch);
      r.d3 = reinterpret_cast<const float4*>((slot_in[d.r3] ? p.pop1 : p.pop0) + (size_t)d.r3 * p.pitch);
    }
    __syncthreads();

    // crossover mask + mutation of the masked genes
    int cnt = 0;
    if (active && !eval_only) {
      const BatchRowShared& r = s_row[gi];
      const int jrand = r.jrand, L = r.L;
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
        const int q = gl + k * G;
        if (q < p.D4) {
          const int j0 = 4 * q;
          unsigned m = 0u;
          if (xo == kBin) {
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
          if (m) {
            const float4 a1 = ld_ro(r.d1 + q), a2 = ld_ro(r.d2 + q), a3 = ld_ro(r.d3 + q);
            if (m & 1u) x[k].x = clip_box(mutate(a1.x, a2.x, a3.x, p.F), p.lo, p.hi);
            if (m & 2u) x[k].y = clip_box(mutate(a1.y, a2.y, a3.y, p.F), p.lo, p.hi);
            if (m & 4u) x[k].z = clip_box(mutate(a1.z, a2.z, a3.z, p.F), p.lo, p.hi);
            if (m & 8u) x[k].w = clip_box(mutate(a1.w, a2.w, a3.w, p.F), p.lo, p.hi);
          }
          cnt += __popc(m);
        }
      }
    }

    // fitness of the trial, reduced over the group
    Acc s{0.0f, 0.0f, 0.0f};
    const int W = min(G, 32);                        // shuffle width
    if (obj == kRosenbrock) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kBatchVmax; ++k) s_first[k][warp] = x[k].x;
      }
      __syncthreads();
      const int gw0 = (gi * G) >> 5;                 // first warp of this group (G >= 32)
      const int gwn = (G + 31) >> 5;                 // warps per group
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
        float nb = __shfl_down_sync(0xFFFFFFFFu, x[k].x, 1, W);
        const float next0 = __shfl_sync(0xFFFFFFFFu, (k + 1 < kBatchVmax) ? x[k + 1].x : 0.0f, 0, W);
        if ((gl & (W - 1)) == W - 1) {
          if (G <= 32) nb = next0;                   // group lane 0, next slot
          else if (warp + 1 < gw0 + gwn) nb = s_first[k][warp + 1];
          else nb = (k + 1 < kBatchVmax) ? s_first[k + 1][gw0] : 0.0f;
        }
        const int q = gl + k * G;
        if (active && q < p.D4) {
          const int j0 = 4 * q;
          if (j0 + 1 < p.D) accum_pair(s, x[k].x, x[k].y);
          if (j0 + 2 < p.D) accum_pair(s, x[k].y, x[k].z);
          if (j0 + 3 < p.D) accum_pair(s, x[k].z, x[k].w);
          if (j0 + 4 < p.D) accum_pair(s, x[k].w, nb);
        }
      }
    } else if (active) {
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
        const int q = gl + k * G;
        if (q < p.D4) {
          const int j0 = 4 * q;
          accum_gene_rt(obj, s, x[k].x, j0, p);
          if (j0 + 1 < p.D) accum_gene_rt(obj, s, x[k].y, j0 + 1, p);
          if (j0 + 2 < p.D) accum_gene_rt(obj, s, x[k].z, j0 + 2, p);
          if (j0 + 3 < p.D) accum_gene_rt(obj, s, x[k].w, j0 + 3, p);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o < W) {
        s.a += __shfl_xor_sync(0xFFFFFFFFu, s.a, o, W);
        s.b += __shfl_xor_sync(0xFFFFFFFFu, s.b, o, W);
        s.c += __shfl_xor_sync(0xFFFFFFFFu, s.c, o, W);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o, W);
      }
    }
    if (G > 32) {
      if (lane == 0) {
        s_red[0][warp] = s.a;
        s_red[1][warp] = s.b;
        s_red[2][warp] = s.c;
        s_red[3][warp] = __int_as_float(cnt);
      }
      __syncthreads();
      if (gl == 0) {
        const int gw0 = (gi * G) >> 5, gwn = G >> 5;
        Acc r{0.0f, 0.0f, 0.0f};
        int c = 0;
        for (int w = 0; w < gwn; ++w) {
          r.a += s_red[0][gw0 + w];
          r.b += s_red[1][gw0 + w];
          r.c += s_red[2][gw0 + w];
          c += __float_as_int(s_red[3][gw0 + w]);
        }
        s = r;
        cnt = c;
      }
    }

    // evaluation only: the parent's fitness and the best key
    if (eval_only && active && gl == 0) {
      float f = finalize_rt(obj, s, p);
      if (f != f) f = __int_as_float(0x7F800000);
      p.fit[i] = f;
      atomicMin(&p.st->best_key, best_key_of(f, i));
    }
    // selection by the group leader
    if (!eval_only && active && gl == 0) {
      BatchRowShared& r = s_row[gi];
      float f = finalize_rt(obj, s, p);
      if (f != f) f = __int_as_float(0x7F800000);
      const int acc = (f < p.fit[i]) ? 1 : 0;
      r.accept = acc;
      slot_out[i] = (uint8_t)(acc ? 1 - r.si : r.si);
      const int Lrow = (xo == kBin) ? cnt : r.L;
      if (acc) {
        p.fit[i] = f;
        atomicMin(&p.st->best_key, best_key_of(f, i));
        atomicAdd(&s_acc, 1ull);
      }
      atomicAdd(&s_msk, (unsigned long long)Lrow);
      if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
      if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
      if (p.dbg_draws) {
        int* o = p.dbg_draws + 5 * (size_t)i;
        o[0] = r.r1; o[1] = r.r2; o[2] = r.r3; o[3] = r.jrand; o[4] = Lrow;
      }
    }
    __syncthreads();
    if (active && !eval_only) {
      const BatchRowShared& r = s_row[gi];
      if (r.accept) {
        float4* out = reinterpret_cast<float4*>((r.si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
#pragma unroll
        for (int k = 0; k < kBatchVmax; ++k) {
          const int q = gl + k * G;
          if (q < p.D4) st_stream(out + q, x[k]);
        }
      }
      if (p.dbg_trial) {
        float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * p.pitch);
#pragma unroll
        for (int k = 0; k < kBatchVmax; ++k) {
          const int q = gl + k * G;
          if (q < p.D4) o[q] = x[k];
        }
      }
    }

    // tile counters; the instance's last tile closes its generation
    if (t == 0) {
      if (s_acc) atomicAdd(&p.st->accepts, s_acc);
      if (s_msk) atomicAdd(&p.st->masked, s_msk);
      __threadfence();
      const unsigned prev = atomicAdd(&p.st->done, 1u);
      if (prev == (unsigned)sI.tiles - 1u) {
        __threadfence();
        const unsigned long long bk = atomicAdd(&p.st->best_key, 0ULL);
        const float bf = from_ordered_bits((uint32_t)(bk >> 32));
        if (eval_only) {
          p.st->best_f = bf;
          p.st->best_gen = gen;
        } else {
          if (bf < p.st->best_f) {
            p.st->best_f = bf;
            p.st->best_gen = gen + 1;
          }
          p.st->gen = gen + 1;
        }
        p.st->done = 0u;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_batch_gen(const BatchInst* insts, const BatchTile* tiles, int ntiles, int grid, bool eval_only,
                             cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  batch_gen_kernel<<<grid, kBatchThreads, 0, s>>>(insts, tiles, ntiles, eval_only ? 1 : 0);
  return cudaGetLastError();
}

__global__ void batch_reset_best_kernel(DevState* states, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    states[k].best_key = ~0ULL;
}

cudaError_t launch_batch_reset_best(DevState* states, int n, cudaStream_t s) {
  batch_reset_best_kernel<<<(n + 255) / 256, 256, 0, s>>>(states, n);
  return cudaGetLastError();
}

}  // namespace de
