// batch_plan.cuh — per-row draws of the batched generation (the row plan)
// and the per-instance close, shared by the plan kernel and the one-launch
// generation of the staged kernel.
#pragma once
#include "draws.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace de {

constexpr int kBatchTableCap = 4096;                // NEC thresholds staged in shared memory

// The draws of row i of instance I: r1, r2, r3 and j_rand (the base rule in
// force) and L (NEC by the threshold table tab, staged in shared memory or,
// when tab is null, read from global memory; exp by the sequential walk).
__device__ __forceinline__ void row_draws(const BatchInst& I, long long gen, int i, const uint32_t* tab,
                                          RowDraws& d, int& Lout) {
  const GenParams& p = I.g;
  const uint32_t g = (uint32_t)gen;
  draw_donors(p, g, i, d);
  int L = 0;
  if (I.xo == kNec) {
    if (p.cr_mode != kCrGeneral) {
      L = (p.cr_mode == kCrZero) ? 1 : p.D;
    } else {
      const uint32_t w = nec_word(p, g, i);
      L = tab ? nec_length_of<true>(p, w, tab) : nec_length_of<false>(p, w, p.nec_tm1);
    }
  } else if (I.xo == kExp) {
    L = exp_walk_length(p, g, i);
  }
  Lout = L;
}

// The plan of row i from its draws: the slot bytes of the row and its
// donors, the parent fitness and the generation parity.
__device__ __forceinline__ RowPlan32 row_plan(const GenParams& p, long long gen, int i, const RowDraws& d, int L) {
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  RowPlan32 pl;
  pl.r1 = d.r1; pl.r2 = d.r2; pl.r3 = d.r3; pl.jrand = d.jrand; pl.L = L;
  pl.slots = (uint32_t)slot_in[i] | ((uint32_t)slot_in[d.r1] << 8) | ((uint32_t)slot_in[d.r2] << 16) |
             ((uint32_t)slot_in[d.r3] << 24);
  pl.fit_i = p.fit[i];
  pl.gpar = (int)(gen & 1);
  return pl;
}

__device__ __forceinline__ RowPlan32 make_row_plan(const BatchInst& I, int i, const uint32_t* tab) {
  const long long gen = I.g.st->gen;
  RowDraws d;
  int L;
  row_draws(I, gen, i, tab, d, L);
  return row_plan(I.g, gen, i, d, L);
}

// The plans of every row of every instance, by plan tiles of 256 rows, for a
// one-launch generation: each CTA takes a contiguous run of tiles (tiles are
// in instance order, so an instance's NEC table is staged in the CTA's
// shared memory `tab` once or twice, not per tile); kThreads threads make one
// or two rows each, the draws of both rows before the gathers of both so
// that their loads are in flight together.
template <int kThreads>
__device__ __forceinline__ void plan_phase(const BatchInst* __restrict__ insts, const BatchTile* __restrict__ ptiles,
                                           int nptiles, RowPlan32* __restrict__ plans, uint32_t* tab) {
  static_assert(kBatchThreadsHost % kThreads == 0 && kBatchThreadsHost / kThreads <= 2,
                "one or two plan rows per thread");
  constexpr int kPer = kBatchThreadsHost / kThreads;
  int cached = -1;
  const int per = (nptiles + (int)gridDim.x - 1) / (int)gridDim.x;
  const int t_end = min(nptiles, ((int)blockIdx.x + 1) * per);
  for (int tile = (int)blockIdx.x * per; tile < t_end; ++tile) {
    const BatchTile tl = ptiles[tile];
    const BatchInst& I = insts[tl.inst];
    const bool tab_smem = (I.xo == kNec) && I.g.nT <= kBatchTableCap;
    if (tl.inst != cached) {                       // uniform over the CTA
      __syncthreads();
      if (tab_smem)
        for (int k = threadIdx.x; k < I.g.nT; k += kThreads) tab[k] = I.g.nec_tm1[k];
      __syncthreads();
      cached = tl.inst;
    }
    const long long gen = I.g.st->gen;
    const int i0 = tl.row0 + threadIdx.x;
    if constexpr (kPer == 2) {
      const int i1 = i0 + kThreads;
      RowDraws d0, d1;
      int L0 = 0, L1 = 0;
      if (i0 < I.g.N) row_draws(I, gen, i0, tab_smem ? tab : nullptr, d0, L0);
      if (i1 < I.g.N) row_draws(I, gen, i1, tab_smem ? tab : nullptr, d1, L1);
      if (i0 < I.g.N) {
        const RowPlan32 a = row_plan(I.g, gen, i0, d0, L0);
        if (i1 < I.g.N) {
          const RowPlan32 b2 = row_plan(I.g, gen, i1, d1, L1);
          plans[I.row_base + i1] = b2;
        }
        plans[I.row_base + i0] = a;
      }
    } else {
      if (i0 < I.g.N) {
        RowDraws d0;
        int L0 = 0;
        row_draws(I, gen, i0, tab_smem ? tab : nullptr, d0, L0);
        plans[I.row_base + i0] = row_plan(I.g, gen, i0, d0, L0);
      }
    }
  }
}

// Grid-wide barrier of a cooperative launch (every CTA resident): an arrival
// counter and a sense word that flips once all CTAs have arrived. The wait is
// bounded by limit_ns of %globaltimer; false if it gave up. Every CTA arrives
// exactly once whether or not it gives up, so the last arrival always resets
// the counter and flips the sense: both are ready for the next launch.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* sense, unsigned nblocks,
                                             unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned s0 = atomicAdd(sense, 0u);
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1u) {
      atomicExch(count, 0u);
      __threadfence();
      atomicExch(sense, s0 ^ 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (atomicAdd(sense, 0u) == s0) {
        if (global_ns() - t0 > limit_ns) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fold a finished generation (or the initial evaluation) into an instance's
// best value / best generation, snapshot its best row and advance it.
__device__ __forceinline__ void close_instance(DevState& st, int eval_only) {
  const float bf = from_ordered_bits((uint32_t)(st.best_key >> 32));
  st.base_row = (int)(uint32_t)(st.best_key & 0xFFFFFFFFull);
  if (eval_only) {
    st.best_f = bf;
    st.best_gen = st.gen;
  } else {
    if (bf < st.best_f) {
      st.best_f = bf;
      st.best_gen = st.gen + 1;
    }
    st.gen = st.gen + 1;
  }
  st.done = 0u;
}

}  // namespace de
