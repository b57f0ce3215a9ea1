// batch_kernel.cu — one generation of many independent DE instances (each
// with its own N, D, objective, crossover, Cr, F, box and Philox instance
// field), in a few launches over all instances:
//
//  1. batch_plan_kernel: one thread per row of every instance draws r1, r2,
//     r3, j_rand and L (NEC through the threshold table staged in shared
//     memory, exp by the sequential walk), and gathers the slot bytes of the
//     row and its donors and the parent fitness into a 32-byte plan. Rows are
//     independent, so the serial draw work of one row never delays another.
//  2. the row kernels: batch_stage_kernel (batch_stage.cu) for exp / NEC
//     rows of D <= 2048 staged through shared memory, batch_span_kernel
//     (batch_span.cuh; one launch per crossover present) for the instances
//     with G <= 32 lanes per row kept in registers, and
//     batch_gen_kernel here for wider rows (CTA tiles of R = 256 / G rows,
//     G = 64, 128 or 256, grid-stride over a tile list grouped by
//     (objective, crossover), longest tiles first). A row's group reads its
//     plan, then issues the parent loads and the donor loads of the masked
//     genes together (one memory round trip), applies Eq. (1) with clipping,
//     reduces the FP32 fitness over the group, selects (strict '<') and
//     stores accepted rows to the other slot buffer.
//  3. batch_close_kernel: one thread per instance folds the generation into
//     its best value / best generation and advances its generation counter.
//
// When every instance is on the staged kernel, the three steps run as one
// cooperative launch instead (batch_stage.cu). With eval_only, the row
// kernels evaluate the parents instead (initial evaluation), so stored and
// trial fitness share one reduction order.
#include <algorithm>

#include "batch_plan.cuh"
#include "draws.cuh"
#include "gen_kernel.cuh"
#include "internal.h"
#include "objectives.cuh"

namespace de {

constexpr int kBatchThreads = 256;
constexpr int kBatchVmax = 16;

// ---------------------------------------------------------------------------
// 1. plans
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchThreads)
batch_plan_kernel(const BatchInst* __restrict__ insts, const BatchTile* __restrict__ ptiles, int nptiles,
                  RowPlan32* __restrict__ plans) {
  __shared__ uint32_t s_tab[kBatchTableCap];
  int cached = -1;
  for (int tile = blockIdx.x; tile < nptiles; tile += gridDim.x) {
    const BatchTile tl = ptiles[tile];
    const BatchInst& I = insts[tl.inst];
    const GenParams& p = I.g;
    const bool tab_smem = (I.xo == kNec) && p.nT <= kBatchTableCap;
    if (tl.inst != cached) {                   // uniform: every thread sees the same tile
      __syncthreads();                         // previous table no longer read
      if (tab_smem)
        for (int k = threadIdx.x; k < p.nT; k += kBatchThreads) s_tab[k] = p.nec_tm1[k];
      __syncthreads();
      cached = tl.inst;
    }
    const int i = tl.row0 + threadIdx.x;
    if (i >= p.N) continue;
    plans[I.row_base + i] = make_row_plan(I, i, tab_smem ? s_tab : nullptr);
  }
}

// ---------------------------------------------------------------------------
// 2. rows
// ---------------------------------------------------------------------------
struct BatchSmem {
  float first[kBatchVmax][kBatchThreads / 32];
  float red[4][kBatchThreads / 32];
  int accept[kBatchThreads / 4];
  int masked[kBatchThreads / 4];
  unsigned long long key[kBatchThreads / 4];
};

// The rows of one tile, specialised for one objective and crossover. Kept
// out of line so that each specialisation is its own compact code: the tile
// list is grouped by (objective, crossover), so the SMs run one
// specialisation at a time and it stays in the instruction cache.
template <int OBJ, int XO>
__device__ __noinline__ void batch_rows(const BatchInst& I, const BatchTile tl, const RowPlan32* __restrict__ plans,
                                        int eval_only, BatchSmem& sm) {
  const GenParams& p = I.g;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = I.group;
  const int gi = t / G, gl = t - gi * G;          // row within the tile, lane within the row's group
  const int i = tl.row0 + gi;
  const bool active = i < p.N;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const int D = p.D, D4 = p.D4;
  const float F = p.F, lo = p.lo, hi = p.hi;

  RowPlan32 pl{};
  if (active) {
    if (eval_only) pl.slots = p.slots[(size_t)(gen & 1) * p.N + i];
    else pl = plans[I.row_base + i];
  }
  const int si = (int)(pl.slots & 0xFFu);
  const float4* xrow = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)(active ? i : 0) * p.pitch);
  const float4* d1 = reinterpret_cast<const float4*>(((pl.slots >> 8) & 0xFFu ? p.pop1 : p.pop0) + (size_t)pl.r1 * p.pitch);
  const float4* d2 = reinterpret_cast<const float4*>(((pl.slots >> 16) & 0xFFu ? p.pop1 : p.pop0) + (size_t)pl.r2 * p.pitch);
  const float4* d3 = reinterpret_cast<const float4*>(((pl.slots >> 24) & 0xFFu ? p.pop1 : p.pop0) + (size_t)pl.r3 * p.pitch);

  // parent row and the donor genes of masked slots, all loads in flight together
  float4 x[kBatchVmax];
  unsigned mk[kBatchVmax];
#pragma unroll
  for (int k = 0; k < kBatchVmax; ++k) {
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
        if (dd < 0) dd += D;                       // (j0 - j_rand) mod D
        if (dd >= pl.L && dd + 3 < D) {
          m = 0u;                                  // the slot lies wholly outside the segment
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            int de = dd + e;
            if (de >= D) de -= D;
            m |= (de < pl.L) ? (1u << e) : 0u;
          }
        }
      }
      m &= (1u << min(4, D - j0)) - 1u;
    }
    mk[k] = m;
  }
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < kBatchVmax; ++k) {
    if (mk[k]) {
      const int q = gl + k * G;
      const float4 a1 = ld_ro(d1 + q), a2 = ld_ro(d2 + q), a3 = ld_ro(d3 + q);
      const unsigned m = mk[k];
      if (m & 1u) x[k].x = clip_box(mutate(a1.x, a2.x, a3.x, F), lo, hi);
      if (m & 2u) x[k].y = clip_box(mutate(a1.y, a2.y, a3.y, F), lo, hi);
      if (m & 4u) x[k].z = clip_box(mutate(a1.z, a2.z, a3.z, F), lo, hi);
      if (m & 8u) x[k].w = clip_box(mutate(a1.w, a2.w, a3.w, F), lo, hi);
      cnt += __popc(m);
    }
  }

  // fitness of the trial (or the parent), reduced over the group
  Acc s{0.0f, 0.0f, 0.0f};
  const int W = min(G, 32);                        // shuffle width
  if constexpr (OBJ == kRosenbrock) {
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) sm.first[k][warp] = x[k].x;
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
        else if (warp + 1 < gw0 + gwn) nb = sm.first[k][warp + 1];
        else nb = (k + 1 < kBatchVmax) ? sm.first[k + 1][gw0] : 0.0f;
      }
      const int q = gl + k * G;
      if (active && q < D4) {
        const int j0 = 4 * q;
        if (j0 + 1 < D) accum_pair(s, x[k].x, x[k].y);
        if (j0 + 2 < D) accum_pair(s, x[k].y, x[k].z);
        if (j0 + 3 < D) accum_pair(s, x[k].z, x[k].w);
        if (j0 + 4 < D) accum_pair(s, x[k].w, nb);
      }
    }
  } else {
    if (active) {
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
            const int q = gl + k * G;
        if (q < D4) {
          const int j0 = 4 * q;
          accum_gene<OBJ>(s, x[k].x, j0, p);
          if (j0 + 1 < D) accum_gene<OBJ>(s, x[k].y, j0 + 1, p);
          if (j0 + 2 < D) accum_gene<OBJ>(s, x[k].z, j0 + 2, p);
          if (j0 + 3 < D) accum_gene<OBJ>(s, x[k].w, j0 + 3, p);
        }
      }
    }
  }
  constexpr int NS = ObjTraits<OBJ>::kSums;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < W) {
      s.a += __shfl_xor_sync(0xFFFFFFFFu, s.a, o, W);
      if (NS > 1) s.b += __shfl_xor_sync(0xFFFFFFFFu, s.b, o, W);
      if (NS > 2) s.c += __shfl_xor_sync(0xFFFFFFFFu, s.c, o, W);
      if (XO == kBin) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o, W);
    }
  }
  if (G > 32) {
    if (lane == 0) {
      sm.red[0][warp] = s.a;
      sm.red[1][warp] = s.b;
      sm.red[2][warp] = s.c;
      sm.red[3][warp] = __int_as_float(cnt);
    }
    __syncthreads();
    if (gl == 0) {
      const int gw0 = (gi * G) >> 5, gwn = G >> 5;
      Acc r{0.0f, 0.0f, 0.0f};
      int c = 0;
      for (int w = 0; w < gwn; ++w) {
        r.a += sm.red[0][gw0 + w];
        r.b += sm.red[1][gw0 + w];
        r.c += sm.red[2][gw0 + w];
        c += __float_as_int(sm.red[3][gw0 + w]);
      }
      s = r;
      cnt = c;
    }
  }

  // decision by the group leader; the tile's counters go to the state once
  if (gl == 0) {
    sm.accept[gi] = 0;
    sm.masked[gi] = 0;
    sm.key[gi] = ~0ull;
  }
  if (active && gl == 0) {
    float f = finalize_fitness<OBJ>(s, p);
    if (f != f) f = __int_as_float(0x7F800000);
    if (eval_only) {
      p.fit[i] = f;
      sm.key[gi] = best_key_of(f, i);
    } else {
      const int acc = (f < pl.fit_i) ? 1 : 0;
      sm.accept[gi] = acc;
      p.slots[(size_t)((gen + 1) & 1) * p.N + i] = (uint8_t)(acc ? 1 - si : si);
      const int Lrow = (XO == kBin) ? cnt : pl.L;
      sm.masked[gi] = Lrow;
      if (acc) {
        p.fit[i] = f;
        sm.key[gi] = best_key_of(f, i);
      }
      if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
      if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
      if (p.dbg_draws) {
        int* o = p.dbg_draws + 5 * (size_t)i;
        o[0] = pl.r1; o[1] = pl.r2; o[2] = pl.r3; o[3] = pl.jrand; o[4] = Lrow;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int R = kBatchThreads / G;
    unsigned long long k = ~0ull, masked = 0, accepts = 0;
    for (int r = 0; r < R; ++r) {
      k = (sm.key[r] < k) ? sm.key[r] : k;
      masked += (unsigned long long)sm.masked[r];
      accepts += (unsigned long long)sm.accept[r];
    }
    if (k != ~0ull) atomicMin(&p.st->best_key, k);
    if (!eval_only) {
      if (accepts) atomicAdd(&p.st->accepts, accepts);
      atomicAdd(&p.st->masked, masked);
    }
  }
  if (active && !eval_only) {
    if (sm.accept[gi]) {
      float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
            const int q = gl + k * G;
        if (q < D4) st_stream(out + q, x[k]);
      }
    }
    if (p.dbg_trial) {
      float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * p.pitch);
#pragma unroll
      for (int k = 0; k < kBatchVmax; ++k) {
            const int q = gl + k * G;
        if (q < D4) o[q] = x[k];
      }
    }
  }
}

template <int OBJ>
__device__ __forceinline__ void batch_rows_xo(int xo, const BatchInst& I, const BatchTile tl,
                                              const RowPlan32* plans, int eval_only, BatchSmem& sm) {
  if (xo == kBin) batch_rows<OBJ, kBin>(I, tl, plans, eval_only, sm);
  else if (xo == kExp) batch_rows<OBJ, kExp>(I, tl, plans, eval_only, sm);
  else batch_rows<OBJ, kNec>(I, tl, plans, eval_only, sm);
}

__global__ void __launch_bounds__(kBatchThreads, 2)
batch_gen_kernel(const BatchInst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                 const RowPlan32* __restrict__ plans, int eval_only) {
  __shared__ BatchSmem sm;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const BatchTile tl = tiles[tile];
    const BatchInst& I = insts[tl.inst];
    const int obj = I.obj, xo = I.xo;                // uniform over the CTA
    switch (obj) {
      case kSphere: batch_rows_xo<kSphere>(xo, I, tl, plans, eval_only, sm); break;
      case kRastrigin: batch_rows_xo<kRastrigin>(xo, I, tl, plans, eval_only, sm); break;
      case kAckley: batch_rows_xo<kAckley>(xo, I, tl, plans, eval_only, sm); break;
      case kRosenbrock: batch_rows_xo<kRosenbrock>(xo, I, tl, plans, eval_only, sm); break;
      case kGriewank: batch_rows_xo<kGriewank>(xo, I, tl, plans, eval_only, sm); break;
      default: batch_rows_xo<kElliptic>(xo, I, tl, plans, eval_only, sm); break;
    }
    __syncthreads();                                 // shared scratch reused by the next tile
  }
}

// ---------------------------------------------------------------------------
// 3. close
// ---------------------------------------------------------------------------
__global__ void batch_close_kernel(DevState* states, int n, int eval_only) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    close_instance(states[k], eval_only);
}

__global__ void batch_reset_best_kernel(DevState* states, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    states[k].best_key = ~0ULL;
}

// The plan kernel is latency-bound (table, then slot bytes and fitness, per
// tile): four times the row kernels' grid keeps more tiles in flight.
static int plan_grid(int nptiles, int grid) { return std::max(1, std::min(nptiles, 4 * grid)); }

cudaError_t launch_batch_plans(const BatchInst* insts, const BatchTile* ptiles, int nptiles, RowPlan32* plans,
                               int grid, cudaStream_t s) {
  batch_plan_kernel<<<plan_grid(nptiles, grid), kBatchThreads, 0, s>>>(insts, ptiles, nptiles, plans);
  return cudaGetLastError();
}

static cudaError_t launch_spans(const BatchInst* insts, const BatchWork& w, const RowPlan32* plans, int eval_only,
                                int grid, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (w.nspans[kBin] > 0 && e == cudaSuccess)
    e = launch_batch_span_bin(insts, w.spans[kBin], w.nspans[kBin], plans, w.ctr + 0, eval_only, grid, s);
  if (w.nspans[kExp] > 0 && e == cudaSuccess)
    e = launch_batch_span_exp(insts, w.spans[kExp], w.nspans[kExp], plans, w.ctr + 2, eval_only, grid, s);
  if (w.nspans[kNec] > 0 && e == cudaSuccess)
    e = launch_batch_span_nec(insts, w.spans[kNec], w.nspans[kNec], plans, w.ctr + 4, eval_only, grid, s);
  if (w.nspans[3] > 0 && e == cudaSuccess)
    e = launch_batch_stage(insts, w.spans[3], w.nspans[3], plans, w.ctr + 6, eval_only, grid, s);
  if (w.nspans[4] > 0 && e == cudaSuccess)
    e = launch_batch_flow(insts, w.spans[4], w.nspans[4], plans, w.ctr + 12, eval_only, grid, s);
  return e;
}

cudaError_t launch_batch_rows(const BatchInst* insts, const BatchWork& w, const RowPlan32* plans, int grid,
                              cudaStream_t s) {
  cudaError_t e = launch_spans(insts, w, plans, 0, grid, s);
  if (e != cudaSuccess) return e;
  if (w.nctiles > 0) batch_gen_kernel<<<grid, kBatchThreads, 0, s>>>(insts, w.ctiles, w.nctiles, plans, 0);
  return cudaGetLastError();
}

cudaError_t launch_batch_generation(const BatchInst* insts, const BatchWork& w, const BatchTile* ptiles,
                                    int nptiles, RowPlan32* plans, DevState* states, int n_inst, int grid,
                                    cudaStream_t s) {
  const int reg = w.nspans[0] + w.nspans[1] + w.nspans[2] + w.nctiles;
  if (reg + w.nspans[3] + w.nspans[4] <= 0) return cudaSuccess;
  // one cooperative launch when every instance is on the staged kernel, or
  // every instance on the streaming kernel
  if (reg + w.nspans[4] == 0 && batch_fused_supported())
    return launch_batch_fused(insts, w.spans[3], w.nspans[3], ptiles, nptiles, plans, states, n_inst, w.ctr + 6,
                              grid, w.wait_ns, s);
  if (reg + w.nspans[3] == 0 && batch_flow_fused_supported())
    return launch_batch_flow_fused(insts, w.spans[4], w.nspans[4], ptiles, nptiles, plans, states, n_inst,
                                   w.ctr + 12, grid, w.wait_ns, s);
  batch_plan_kernel<<<plan_grid(nptiles, grid), kBatchThreads, 0, s>>>(insts, ptiles, nptiles, plans);
  cudaError_t e = launch_spans(insts, w, plans, 0, grid, s);
  if (e != cudaSuccess) return e;
  if (w.nctiles > 0) batch_gen_kernel<<<grid, kBatchThreads, 0, s>>>(insts, w.ctiles, w.nctiles, plans, 0);
  batch_close_kernel<<<(n_inst + 255) / 256, 256, 0, s>>>(states, n_inst, 0);
  return cudaGetLastError();
}

cudaError_t launch_batch_evaluate(const BatchInst* insts, const BatchWork& w, DevState* states, int first_inst,
                                  int n_inst, int grid, cudaStream_t s) {
  batch_reset_best_kernel<<<(n_inst + 255) / 256, 256, 0, s>>>(states + first_inst, n_inst);
  cudaError_t e = launch_spans(insts, w, nullptr, 1, grid, s);
  if (e != cudaSuccess) return e;
  if (w.nctiles > 0) batch_gen_kernel<<<grid, kBatchThreads, 0, s>>>(insts, w.ctiles, w.nctiles, nullptr, 1);
  batch_close_kernel<<<(n_inst + 255) / 256, 256, 0, s>>>(states + first_inst, n_inst, 1);
  return cudaGetLastError();
}

}  // namespace de
