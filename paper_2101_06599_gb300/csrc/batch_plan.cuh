// batch_plan.cuh — per-row draws of the batched generation (the row plan)
// and the per-instance close, shared by the plan kernel and the one-launch
// generation of the staged kernel.
#pragma once
#include "draws.cuh"
#include "internal.h"

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
