// batch_flow.cu — the streaming row kernel of the batched generation for the
// segment crossovers (sequential exp, Alg. 8, and NEC, Alg. 9 with Eq. 9),
// rows of any length.
//
// One warp per row. The row is walked in chunks of 32 x kFlowU float4 slots
// (lane l holds slots q0 + l + 32 u, u < kFlowU; a u none of whose slots is
// in the row is skipped by the whole warp) loaded straight into registers,
// and the next chunk (of the same row, or the first chunk of the next row of
// the span) is loaded while the current one is processed, so every warp
// always has a chunk of loads in flight. The donor slots of the next row's
// segment are copied into shared memory (cp.async) at the same time. Per row:
//   - the masked genes are the circular segment [j_rand, j_rand + L) mod D,
//     at most two runs of slots. When the runs cover at most 32 slots, lane k
//     takes the three donor float4s of the k-th segment slot and computes its
//     mutant clip(x_r1 + F (x_r2 - x_r3)) (Eq. 1, each operation rounded once)
//     and mask bits, and the lane holding that slot in a chunk takes them by
//     shuffle, only where the segment meets the chunk. Longer segments take
//     the mask of every slot and read their donors slot by slot;
//   - the objective is summed in the canonical order of batch_span.cuh: lane
//     l is virtual lane l (slots l, l + 32, ... in gene order), then the
//     butterfly over strides 16 .. 1; fitness values, selections and
//     trajectories are bit-identical to every row kernel with at most 32
//     lanes per row;
//   - the strict '<' selection against the plan's parent fitness; an
//     accepted row goes to the other slot buffer, from the registers when the
//     row is one chunk (D <= 512), else chunk by chunk again (those parent
//     reads come from L2: the row was read a moment before).
// Work comes from a span list (up to 32 consecutive rows of one instance per
// span, taken from a global queue); the next span's index, descriptor and
// plans are fetched while the current span runs.
//
// The FUSED instantiation is a whole generation of every instance in one
// cooperative launch, as the staged kernel's: the plans of every row, a
// bounded grid barrier, the rows, and the close of every instance by the last
// warp to finish.
#include <algorithm>
#include <cstring>

#include "batch_plan.cuh"
#include "internal.h"
#include "objectives.cuh"
#include "ptx.cuh"

namespace de {

namespace {

constexpr int kFlowWarps = 8;
constexpr int kFlowThreads = 32 * kFlowWarps;
constexpr int kFlowU = 4;                           // float4 slots per lane per chunk
constexpr int kFlowChunk = 32 * kFlowU;             // slots per chunk
constexpr unsigned kFull = 0xFFFFFFFFu;

// Mask bits of slot q (genes 4q .. 4q+3, bit e = gene 4q + e): the genes of
// the circular segment [jrand, jrand + L) mod D.
__device__ __forceinline__ unsigned seg_mask(int q, int D, int jrand, int L) {
  const int j0 = 4 * q;
  int dd = j0 - jrand;
  if (dd < 0) dd += D;                              // (j0 - j_rand) mod D
  unsigned m = 0u;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int de = dd + e;
    if (de >= D) de -= D;
    m |= (de < L) ? (1u << e) : 0u;
  }
  return m & ((1u << min(4, D - j0)) - 1u);        // padding genes never cross
}

__device__ __forceinline__ float4 mutant4(const float4 a1, const float4 a2, const float4 a3, float F, float lo,
                                          float hi) {
  return make_float4(clip_box(mutate(a1.x, a2.x, a3.x, F), lo, hi), clip_box(mutate(a1.y, a2.y, a3.y, F), lo, hi),
                     clip_box(mutate(a1.z, a2.z, a3.z, F), lo, hi), clip_box(mutate(a1.w, a2.w, a3.w, F), lo, hi));
}

__device__ __forceinline__ void apply_bits(float4& x, const float4 v, unsigned m) {
  if (m & 1u) x.x = v.x;
  if (m & 2u) x.y = v.y;
  if (m & 4u) x.z = v.z;
  if (m & 8u) x.w = v.w;
}

// What a row needs beyond its parent slots.
struct FlowRow {
  int i, si, jrand, L;
  float fit_i;
  // the segment: run A = slots qa .. qa + na - 1, run B = slots 0 .. nb - 1
  int qa, na, nb;
  bool fast;                                        // lane k < na + nb holds segment slot k
  float4 v;                                         // that slot's mutant values
  unsigned m;                                       // and mask bits
};

// A warp's span buffers in shared memory: the plans and instance descriptor
// of the span being processed and of the next one (copied while the current
// one runs).
constexpr int kFlowInstWords = (int)(sizeof(BatchInst) / 16);
static_assert(sizeof(BatchInst) % 16 == 0, "instance descriptor copied as uint4");
struct __align__(16) FlowSmem {
  RowPlan32 plan[2][32];
  uint4 inst[2][kFlowInstWords];
  BatchSpan span[2];
  float4 don[2][3][32];                             // donor slots of the segment of rows r and r + 1
};

__device__ __forceinline__ const BatchInst& flow_inst(const FlowSmem& w, int b) {
  return *reinterpret_cast<const BatchInst*>(w.inst[b]);
}

// Instance parameters a row needs, read once per span.
struct FlowInst {
  const float* pop0;
  const float* pop1;
  float* fit;
  uint8_t* slot_out;
  size_t pitch;
  int D, D4, nch;
  float F, lo, hi;
};

__device__ __forceinline__ const float4* row_ptr(const FlowInst& I, int i, int si) {
  return reinterpret_cast<const float4*>((si ? I.pop1 : I.pop0) + (size_t)i * I.pitch);
}

__device__ __forceinline__ void load_chunk(float4 (&a)[kFlowU], const float4* x, int q0, int D4, int lane) {
#pragma unroll
  for (int u = 0; u < kFlowU; ++u) {
    if (q0 + 32 * u >= D4) break;                   // warp-uniform
    const int q = q0 + lane + 32 * u;
    a[u] = (q < D4) ? ld_stream(x + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

__device__ __forceinline__ void donor_ptrs(const FlowInst& I, const RowPlan32& pl, const float4*& d1,
                                           const float4*& d2, const float4*& d3) {
  d1 = row_ptr(I, pl.r1, (int)((pl.slots >> 8) & 0xFFu));
  d2 = row_ptr(I, pl.r2, (int)((pl.slots >> 16) & 0xFFu));
  d3 = row_ptr(I, pl.r3, (int)((pl.slots >> 24) & 0xFFu));
}

// The masked genes of the chunk at q0 replaced by their mutants (pl: the
// row's plan, read only by the path for long segments).
__device__ __forceinline__ void patch_chunk(float4 (&a)[kFlowU], const FlowInst& I, const FlowRow& R,
                                            const RowPlan32& pl, int q0, int lane) {
  if (R.fast) {
#pragma unroll
    for (int u = 0; u < kFlowU; ++u) {
      const int w0 = q0 + 32 * u;                   // slots w0 .. w0 + 31 of this u
      if (w0 >= I.D4) break;                        // warp-uniform
      const bool hit = (w0 < R.qa + R.na && w0 + 32 > R.qa) || (w0 < R.nb);
      if (hit) {                                    // warp-uniform
        const int q = w0 + lane;
        const int k = (q >= R.qa && q < R.qa + R.na) ? q - R.qa : (q < R.nb ? R.na + q : -1);
        float4 v;
        v.x = __shfl_sync(kFull, R.v.x, k & 31);
        v.y = __shfl_sync(kFull, R.v.y, k & 31);
        v.z = __shfl_sync(kFull, R.v.z, k & 31);
        v.w = __shfl_sync(kFull, R.v.w, k & 31);
        const unsigned m = __shfl_sync(kFull, R.m, k & 31);
        if (k >= 0) apply_bits(a[u], v, m);
      }
    }
  } else {
    const float4 *d1, *d2, *d3;
    donor_ptrs(I, pl, d1, d2, d3);
#pragma unroll
    for (int u = 0; u < kFlowU; ++u) {
      if (q0 + 32 * u >= I.D4) break;               // warp-uniform
      const int q = q0 + lane + 32 * u;
      if (q < I.D4) {
        const unsigned m = seg_mask(q, I.D, R.jrand, R.L);
        if (m) apply_bits(a[u], mutant4(ld_ro(d1 + q), ld_ro(d2 + q), ld_ro(d3 + q), I.F, I.lo, I.hi), m);
      }
    }
  }
}

// The objective's terms of the chunk at q0 added to s in the canonical order.
// Rosenbrock: the pair of slot q's last gene with slot q + 1's first is taken
// by shuffle; for lane 31's last slot of the chunk it is kept pending (carry)
// and added at the start of the next chunk, before any later term of the lane.
template <int OBJ>
__device__ __forceinline__ void sum_chunk(Acc& s, const float4 (&a)[kFlowU], const FlowInst& I, const GenParams& p,
                                          int q0, int lane, float& carry, bool& pending) {
  if constexpr (OBJ == kRosenbrock) {
    const float first = __shfl_sync(kFull, a[0].x, 0);
    if (pending) {                                  // lane 31 only
      accum_pair(s, carry, first);
      pending = false;
    }
#pragma unroll
    for (int u = 0; u < kFlowU; ++u) {
      if (q0 + 32 * u >= I.D4) break;               // warp-uniform
      const float nl = __shfl_down_sync(kFull, a[u].x, 1);
      const float nw = (u + 1 < kFlowU) ? __shfl_sync(kFull, a[(u + 1) % kFlowU].x, 0) : 0.0f;
      const float nb = (lane == 31) ? nw : nl;
      const int q = q0 + lane + 32 * u;
      if (q < I.D4) {
        const int j0 = 4 * q;
        if (j0 + 1 < I.D) accum_pair(s, a[u].x, a[u].y);
        if (j0 + 2 < I.D) accum_pair(s, a[u].y, a[u].z);
        if (j0 + 3 < I.D) accum_pair(s, a[u].z, a[u].w);
        if (j0 + 4 < I.D) {
          if (lane == 31 && u + 1 == kFlowU) {
            carry = a[u].w;
            pending = true;
          } else {
            accum_pair(s, a[u].w, nb);
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < kFlowU; ++u) {
      if (q0 + 32 * u >= I.D4) break;               // warp-uniform
      const int q = q0 + lane + 32 * u;
      if (q < I.D4) {
        const int j0 = 4 * q;
        accum_gene<OBJ>(s, a[u].x, j0, p);
        if (j0 + 4 <= I.D) {
          accum_gene<OBJ>(s, a[u].y, j0 + 1, p);
          accum_gene<OBJ>(s, a[u].z, j0 + 2, p);
          accum_gene<OBJ>(s, a[u].w, j0 + 3, p);
        } else {
          if (j0 + 1 < I.D) accum_gene<OBJ>(s, a[u].y, j0 + 1, p);
          if (j0 + 2 < I.D) accum_gene<OBJ>(s, a[u].z, j0 + 2, p);
        }
      }
    }
  }
}

// The segment of a row at slot level: run A = slots qa .. qa + na - 1, run
// B = slots 0 .. nb - 1 (the wrap); fast when the runs are disjoint and cover
// at most 32 slots (one per lane).
__device__ __forceinline__ void seg_runs(int D, int jrand, int L, int& qa, int& na, int& nb, bool& fast) {
  const int eA = min(jrand + L, D);                 // run A: genes jrand .. eA - 1
  const int eB = jrand + L - D;                     // run B: genes 0 .. eB - 1
  qa = jrand >> 2;
  na = ((eA - 1) >> 2) - qa + 1;
  nb = eB > 0 ? ((eB - 1) >> 2) + 1 : 0;
  fast = (na + nb <= 32) && (nb <= qa);
}

// Copy the donor slots of row pl's segment into don (lane k: the k-th
// segment slot of each donor) with cp.async; nothing for long segments.
// The caller commits the group.
__device__ __forceinline__ void prefetch_donors(float4 (&don)[3][32], const FlowInst& I, const RowPlan32& pl,
                                                int lane) {
  int qa, na, nb;
  bool fast;
  seg_runs(I.D, pl.jrand, pl.L, qa, na, nb, fast);
  if (fast && lane < na + nb) {
    const int q = lane < na ? qa + lane : lane - na;
    const float4 *d1, *d2, *d3;
    donor_ptrs(I, pl, d1, d2, d3);
    ca16_g2s(smem_u32(&don[0][lane]), d1 + q);
    ca16_g2s(smem_u32(&don[1][lane]), d2 + q);
    ca16_g2s(smem_u32(&don[2][lane]), d3 + q);
  }
}

// Row r of the span from its plan pl (shared memory): the segment, its
// mutants from the donor slots already copied into don.
__device__ __forceinline__ void start_row(FlowRow& R, const FlowInst& I, const RowPlan32& pl,
                                          const float4 (&don)[3][32], int row0, int r, int lane, int eval_only) {
  R.i = row0 + r;
  R.si = (int)(pl.slots & 0xFFu);
  R.fast = true;
  R.na = 0;
  R.nb = 0;
  R.qa = 0;
  R.m = 0u;
  R.v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (eval_only) return;
  R.jrand = pl.jrand;
  R.L = pl.L;
  R.fit_i = pl.fit_i;
  seg_runs(I.D, R.jrand, R.L, R.qa, R.na, R.nb, R.fast);
  if (R.fast && lane < R.na + R.nb) {
    const int q = lane < R.na ? R.qa + lane : lane - R.na;
    R.m = seg_mask(q, I.D, R.jrand, R.L);
    R.v = mutant4(don[0][lane], don[1][lane], don[2][lane], I.F, I.lo, I.hi);
  }
}

// Where a warp is in its span: job (row r, chunk c), the running sums of row
// r, and the span's counters.
struct FlowState {
  int r, c;
  Acc s;
  float carry;
  bool pending;
  unsigned long long kmin, masked;
  unsigned accepts;
  FlowRow R;
};

// The objective's terms of a chunk, for the instance's objective.
__device__ __forceinline__ void sum_chunk_any(int obj, Acc& s, const float4 (&a)[kFlowU], const FlowInst& I,
                                              const GenParams& p, int q0, int lane, float& carry, bool& pending) {
  switch (obj) {
    case kSphere: sum_chunk<kSphere>(s, a, I, p, q0, lane, carry, pending); break;
    case kRastrigin: sum_chunk<kRastrigin>(s, a, I, p, q0, lane, carry, pending); break;
    case kAckley: sum_chunk<kAckley>(s, a, I, p, q0, lane, carry, pending); break;
    case kRosenbrock: sum_chunk<kRosenbrock>(s, a, I, p, q0, lane, carry, pending); break;
    case kGriewank: sum_chunk<kGriewank>(s, a, I, p, q0, lane, carry, pending); break;
    default: sum_chunk<kElliptic>(s, a, I, p, q0, lane, carry, pending); break;
  }
}

// The row value from the 32 virtual lanes' sums: the butterfly over strides
// 16 .. 1, then the objective's final combine (NaN counts as +inf).
template <int OBJ>
__device__ __forceinline__ float row_value(Acc t, const GenParams& p) {
  constexpr int NS = ObjTraits<OBJ>::kSums;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t.a += __shfl_xor_sync(kFull, t.a, o);
    if (NS > 1) t.b += __shfl_xor_sync(kFull, t.b, o);
    if (NS > 2) t.c += __shfl_xor_sync(kFull, t.c, o);
  }
  float f = finalize_fitness<OBJ>(t, p);
  if (f != f) f = __int_as_float(0x7F800000);
  return f;
}

__device__ __noinline__ float row_value_any(int obj, Acc t, const GenParams& p) {
  switch (obj) {
    case kSphere: return row_value<kSphere>(t, p);
    case kRastrigin: return row_value<kRastrigin>(t, p);
    case kAckley: return row_value<kAckley>(t, p);
    case kRosenbrock: return row_value<kRosenbrock>(t, p);
    case kGriewank: return row_value<kGriewank>(t, p);
    default: return row_value<kElliptic>(t, p);
  }
}

// One job: the next job's loads into nxt, then chunk c of row r from cur,
// and the row's value, selection and store after its last chunk.
__device__ __forceinline__ void flow_job(int obj, FlowState& st, float4 (&cur)[kFlowU], float4 (&nxt)[kFlowU],
                                         FlowSmem& w, const FlowInst& I, const GenParams& p, const RowPlan32* pls,
                                         int rows, int row0, int eval_only, int lane) {
  {
    int rn = st.r, cn = st.c + 1;
    if (cn == I.nch) {
      rn = st.r + 1;
      cn = 0;
    }
    if (rn < rows) {
      const int sn = (int)(pls[rn].slots & 0xFFu);
      load_chunk(nxt, row_ptr(I, row0 + rn, sn), cn * kFlowChunk, I.D4, lane);
      if (cn == 0 && !eval_only) prefetch_donors(w.don[rn & 1], I, pls[rn], lane);
    }
    ca_commit();                                    // one group per job (possibly empty)
  }
  FlowRow& R = st.R;
  const RowPlan32& pl = pls[st.r];
  if (st.c == 0) {
    ca_wait_prior();                                // this row's donor copies (all but the group just made)
    __syncwarp();
    start_row(R, I, pl, w.don[st.r & 1], row0, st.r, lane, eval_only);
    st.s = Acc{0.0f, 0.0f, 0.0f};
    st.pending = false;
  }
  const int q0 = st.c * kFlowChunk;
  if (!eval_only) patch_chunk(cur, I, R, pl, q0, lane);
  sum_chunk_any(obj, st.s, cur, I, p, q0, lane, st.carry, st.pending);
  if (st.c + 1 < I.nch) {
    ++st.c;
    return;
  }
  const float f = row_value_any(obj, st.s, p);
  const int i = R.i;
  st.c = 0;
  ++st.r;
  if (eval_only) {
    if (lane == 0) {
      I.fit[i] = f;
      const unsigned long long key = best_key_of(f, i);
      st.kmin = key < st.kmin ? key : st.kmin;
    }
    return;
  }
  const bool acc = f < R.fit_i;                     // the same in every lane
  if (lane == 0) {
    I.slot_out[i] = (uint8_t)(acc ? 1 - R.si : R.si);
    st.masked += (unsigned long long)R.L;
    if (acc) {
      st.accepts += 1u;
      I.fit[i] = f;
      const unsigned long long key = best_key_of(f, i);
      st.kmin = key < st.kmin ? key : st.kmin;
    }
    if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
    if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
    if (p.dbg_draws) {
      int* o = p.dbg_draws + 5 * (size_t)i;
      o[0] = pl.r1; o[1] = pl.r2; o[2] = pl.r3; o[3] = R.jrand; o[4] = R.L;
    }
  }
  // the trial to the other slot buffer (accepted) and to the test hook's buffer
#pragma unroll 1
  for (int o = 0; o < 2; ++o) {
    float4* out = (o == 0) ? (acc ? reinterpret_cast<float4*>((R.si ? p.pop0 : p.pop1) + (size_t)i * I.pitch) : nullptr)
                           : (p.dbg_trial ? reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * I.pitch) : nullptr);
    if (!out) continue;                             // warp-uniform
    if (I.nch == 1) {
#pragma unroll
      for (int u = 0; u < kFlowU; ++u) {
        if (32 * u >= I.D4) break;                  // warp-uniform
        const int q = lane + 32 * u;
        if (q < I.D4) st_stream(out + q, cur[u]);
      }
    } else {
      // cur is free (this job's chunk is summed): it takes the row again
      const float4* x = row_ptr(I, i, R.si);
#pragma unroll 1
      for (int q1 = 0; q1 < I.D4; q1 += kFlowChunk) {
        load_chunk(cur, x, q1, I.D4, lane);
        patch_chunk(cur, I, R, pl, q1, lane);
#pragma unroll
        for (int u = 0; u < kFlowU; ++u) {
          if (q1 + 32 * u >= I.D4) break;           // warp-uniform
          const int q = q1 + lane + 32 * u;
          if (q < I.D4) st_stream(out + q, cur[u]);
        }
      }
    }
  }
}

// The rows of the span in buffer b of w, then its counters into the
// instance state.
__device__ __forceinline__ void flow_span(FlowSmem& w, int b, int eval_only) {
  const int lane = threadIdx.x & 31;
  const GenParams& p = flow_inst(w, b).g;
  const int obj = flow_inst(w, b).obj;
  const long long gen = p.st->gen;
  FlowInst I;
  I.pop0 = p.pop0;
  I.pop1 = p.pop1;
  I.fit = p.fit;
  I.slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  I.pitch = (size_t)p.pitch;
  I.D = p.D;
  I.D4 = p.D4;
  I.nch = (p.D4 + kFlowChunk - 1) / kFlowChunk;
  I.F = p.F;
  I.lo = p.lo;
  I.hi = p.hi;
  const int rows = w.span[b].rows, row0 = w.span[b].row0;
  const RowPlan32* pls = w.plan[b];

  FlowState st;
  st.r = 0;
  st.c = 0;
  st.s = Acc{0.0f, 0.0f, 0.0f};
  st.carry = 0.0f;
  st.pending = false;
  st.kmin = ~0ull;
  st.masked = 0ull;
  st.accepts = 0u;
  float4 A[kFlowU], B[kFlowU];
  load_chunk(A, row_ptr(I, row0, (int)(pls[0].slots & 0xFFu)), 0, I.D4, lane);
  if (!eval_only) prefetch_donors(w.don[0], I, pls[0], lane);
  ca_commit();
  // one copy of the job code (two alternating copies cost more in instruction
  // fetch than they save): the prefetched chunk moves into A after each job
  while (st.r < rows) {
    flow_job(obj, st, A, B, w, I, p, pls, rows, row0, eval_only, lane);
#pragma unroll
    for (int u = 0; u < kFlowU; ++u) A[u] = B[u];
  }
  // every lane's copies have landed before the buffers are reused
  ca_wait_all();
  __syncwarp();

  // the span's counters
  unsigned long long kmin = st.kmin, masked = st.masked;
  unsigned accepts = st.accepts;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ko = __shfl_xor_sync(kFull, kmin, o);
    kmin = ko < kmin ? ko : kmin;
    masked += __shfl_xor_sync(kFull, masked, o);
    accepts += __shfl_xor_sync(kFull, accepts, o);
  }
  if (lane == 0) {
    if (kmin != ~0ull) atomicMin(&p.st->best_key, kmin);
    if (!eval_only) {
      if (accepts) atomicAdd(&p.st->accepts, (unsigned long long)accepts);
      atomicAdd(&p.st->masked, masked);
    }
  }
}

// Take the next span from the queue into buffer b: its descriptor (read
// now), its instance descriptor and its plans (copied asynchronously; when
// evaluating, each row's slot byte instead). Returns false when the queue is
// empty.
__device__ __forceinline__ bool take_span(FlowSmem& w, int b, const BatchInst* __restrict__ insts,
                                          const BatchSpan* __restrict__ spans, int nspans,
                                          const RowPlan32* __restrict__ plans, unsigned* ctr, int eval_only,
                                          int lane) {
  unsigned q = 0u;
  if (lane == 0) q = atomicAdd(&ctr[0], 1u);
  q = __shfl_sync(kFull, q, 0);
  if (q >= (unsigned)nspans) return false;
  const BatchSpan sp = spans[q];
  if (lane == 0) w.span[b] = sp;
  if (lane < kFlowInstWords)
    ca16_g2s(smem_u32(&w.inst[b][lane]), reinterpret_cast<const uint4*>(insts + sp.inst) + lane);
  if (lane < sp.rows) {
    if (eval_only) {
      const GenParams& g = insts[sp.inst].g;
      RowPlan32 pl = {};
      pl.slots = g.slots[(size_t)(g.st->gen & 1) * g.N + sp.row0 + lane];
      w.plan[b][lane] = pl;
    } else {
      const uint4* src = reinterpret_cast<const uint4*>(plans + sp.plan0 + lane);
      const uint32_t dst = smem_u32(&w.plan[b][lane]);
      ca16_g2s(dst, src);
      ca16_g2s(dst + 16u, src + 1);
    }
  }
  ca_commit();
  return true;
}

// ctr[0]: next span to take; ctr[1]: warps finished (the last one resets
// both); FUSED: ctr[2], ctr[3] the grid barrier (see batch_stage.cu for the
// whole-generation argument, which holds here unchanged).
template <bool FUSED>
__global__ void __launch_bounds__(kFlowThreads, 2)
batch_flow_kernel(const BatchInst* __restrict__ insts, const BatchSpan* __restrict__ spans, int nspans,
                  RowPlan32* __restrict__ plans, unsigned* ctr, int eval_only, const BatchTile* __restrict__ ptiles,
                  int nptiles, DevState* states, int n_inst, unsigned long long wait_ns) {
  extern __shared__ __align__(16) unsigned char flow_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  FlowSmem& w = reinterpret_cast<FlowSmem*>(flow_smem)[warp];
  bool go = true;
  if constexpr (FUSED) {
    // the span buffers are free until the rows: the NEC tables go there
    plan_phase<kFlowThreads>(insts, ptiles, nptiles, plans, reinterpret_cast<uint32_t*>(flow_smem));
    go = grid_barrier(&ctr[2], &ctr[3], gridDim.x, wait_ns);
    if (!go && threadIdx.x == 0) atomicExch(&states[0].error, 4u);   // DE_ETIMEOUT
    __syncthreads();
  }
  if (go) {
    int b = 0;
    bool have = take_span(w, b, insts, spans, nspans, plans, ctr, eval_only, lane);
    while (have) {
      ca_wait_all();
      __syncwarp();
      // the next span travels while this one runs
      const bool next = take_span(w, b ^ 1, insts, spans, nspans, plans, ctr, eval_only, lane);
      flow_span(w, b, eval_only);
      __syncwarp();
      b ^= 1;
      have = next;
    }
  }
  ca_wait_all();
  unsigned done = 0u;
  if (lane == 0) {
    __threadfence();
    done = atomicAdd(&ctr[1], 1u);
  }
  done = __shfl_sync(kFull, done, 0);
  if (done == gridDim.x * kFlowWarps - 1u) {         // the last warp of the launch
    __threadfence();
    if (FUSED)
      for (int k = lane; k < n_inst; k += 32) close_instance(states[k], 0);
    __syncwarp();
    if (lane == 0) {
      ctr[0] = 0u;
      ctr[1] = 0u;
      __threadfence();
    }
  }
}

int g_flow_ctas_per_sm = 2;
int g_flow_fused_ctas_per_sm = 0;

}  // namespace

size_t batch_flow_smem() {
  return std::max((size_t)kFlowWarps * sizeof(FlowSmem), (size_t)kBatchTableCap * sizeof(uint32_t));
}

cudaError_t prepare_batch_flow() {
  cudaError_t e = cudaFuncSetAttribute(batch_flow_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_flow_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_flow_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_flow_smem());
  int n = 0, m = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_flow_kernel<false>, kFlowThreads, batch_flow_smem());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, batch_flow_kernel<true>, kFlowThreads, batch_flow_smem());
  if (e == cudaSuccess && n > 0) g_flow_ctas_per_sm = n;
  if (e == cudaSuccess) g_flow_fused_ctas_per_sm = m;
  return e;
}

bool batch_flow_fused_supported() { return g_flow_fused_ctas_per_sm > 0; }

// grid: the row kernels' grid of two CTAs per SM; this kernel fills every SM
// with as many CTAs as fit.
cudaError_t launch_batch_flow(const BatchInst* insts, const BatchSpan* spans, int nspans, const RowPlan32* plans,
                              unsigned* ctr, int eval_only, int grid, cudaStream_t s) {
  const int g = std::max(1, grid / 2) * g_flow_ctas_per_sm;
  batch_flow_kernel<false><<<g, kFlowThreads, batch_flow_smem(), s>>>(insts, spans, nspans, const_cast<RowPlan32*>(plans), ctr,
                                                       eval_only, nullptr, 0, nullptr, 0, 0ull);
  return cudaGetLastError();
}

// One generation of every instance in one cooperative launch (every instance
// on this kernel). ctr: 4 counters (queue, done, barrier arrivals, sense).
cudaError_t launch_batch_flow_fused(const BatchInst* insts, const BatchSpan* spans, int nspans,
                                    const BatchTile* ptiles, int nptiles, RowPlan32* plans, DevState* states,
                                    int n_inst, unsigned* ctr, int grid, unsigned long long wait_ns,
                                    cudaStream_t s) {
  if (g_flow_fused_ctas_per_sm <= 0) return cudaErrorNotSupported;
  if (wait_ns == 0ull) wait_ns = kWaitLimitNs;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(std::max(1, grid / 2) * g_flow_fused_ctas_per_sm));
  cfg.blockDim = dim3(kFlowThreads);
  cfg.dynamicSmemBytes = batch_flow_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_flow_kernel<true>, insts, spans, nspans, plans, ctr, 0, ptiles, nptiles,
                            states, n_inst, wait_ns);
}

}  // namespace de
