// batch_stage.cu — the row kernel of the batched generation for the
// segment crossovers (sequential exp, Alg. 8, and NEC, Alg. 9 with Eq. 9)
// on instances whose rows hold at most 512 float4 slots (D <= 2048).
//
// Each warp is a two-stage pipeline over passes: a pass is up to 32
// consecutive rows of one instance holding at most 512 float4 slots (8 KB).
// While the warp processes pass p from shared memory, the 128-bit loads of
// pass p + 1 are in flight into registers (16 float4 per lane) and the donor
// genes of p + 1's masked segments [j_rand, j_rand + L) mod D travel into
// shared memory by cp.async; at the top of the next step the registers are
// stored into the pass buffer and the warp moves on. The row code is small
// rolled loops over shared memory, so it stays in the instruction cache.
//
// Rows of a pass are processed G lanes per row, 32 / G rows at a time
// (G = 4, 8, 16 or 32, per instance). The FP32 fitness is summed in the
// canonical order of batch_span.cuh (32 virtual lanes, virtual lane v summing
// the genes of slots v, v + 32, ... in order, then a butterfly 16 .. 1), so
// every G, and the register kernel, give bit-identical values. Then:
//   1. the masked genes: v = clip(x_r1 + F (x_r2 - x_r3)) (Eq. 1) written over
//      the parent's genes in shared memory;
//   2. the fitness of the trial, reduced over the group;
//   3. the strict '<' selection; an accepted row is stored from shared memory
//      to the other slot buffer.
//
// Work comes from the span list (up to 32 rows of one instance per span,
// taken from a global queue). A span's plans and instance descriptor are
// copied into one of three rotating shared buffers one span ahead, so no
// global read sits between two passes; the generation parity comes with the
// row plans. The grid fills every SM with as many CTAs as fit (3 x 4 warps).
//
// The FUSED instantiation is a whole generation of every instance in one
// cooperative launch: the row plans (as batch_plan_kernel), a bounded grid
// barrier, the rows, and the close of every instance by the last warp.
#include <algorithm>
#include <cstring>

#include "batch_plan.cuh"
#include "draws.cuh"
#include "internal.h"
#include "objectives.cuh"
#include "ptx.cuh"

namespace de {

namespace {

constexpr int kPwWarps = 4;                         // warps per CTA
constexpr int kPwThreads = 32 * kPwWarps;
constexpr int kPassSlots = 512;                     // float4 slots of one pass (8 KB)
constexpr int kPassVec = kPassSlots / 32;           // float4 per lane in flight
constexpr int kDonCap = 128;                        // donor genes of one pass in shared memory
constexpr int kDonRowCap = 64;                      // longer segments read their donors from global memory
constexpr int kInstWords = (int)(sizeof(BatchInst) / 16);
static_assert(sizeof(BatchInst) % 16 == 0, "instance descriptor copied as uint4");
static_assert(sizeof(RowPlan32) == 32, "plan copied as two uint4");

struct __align__(16) PassSmem {
  float4 buf[kPassSlots];                           // the pass being processed, rows back to back
  float don[2][3][kDonCap];                         // donor genes of a pass, [pass buffer][donor][gene]
  RowPlan32 plan[3][32];                            // plans of three spans
  uint4 inst[3][kInstWords];                        // their instance descriptors
  int dbase[2][32];                                 // first donor gene of each row of a pass, -1: global
};

struct Pass {
  int pb;        // span buffer
  int row0;      // the span's first row in its instance
  int li0, n;    // rows li0 .. li0 + n - 1 of the span
  int last;      // last pass of its span
};

__device__ __forceinline__ const BatchInst& inst_of(const PassSmem& w, int pb) {
  return *reinterpret_cast<const BatchInst*>(w.inst[pb]);
}

__device__ __forceinline__ void ca4_g2s(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

// Start copying a span's instance descriptor and plans into span buffer pb.
__device__ __forceinline__ void prefetch_span(PassSmem& w, int pb, const BatchSpan& sp, const BatchInst* insts,
                                              const RowPlan32* plans, int eval_only, int lane) {
  if (lane < kInstWords)
    ca16_g2s(smem_u32(&w.inst[pb][lane]), reinterpret_cast<const uint4*>(insts + sp.inst) + lane);
  if (!eval_only && lane < sp.rows) {
    const uint4* src = reinterpret_cast<const uint4*>(plans + sp.plan0 + lane);
    const uint32_t dst = smem_u32(&w.plan[pb][lane]);
    ca16_g2s(dst, src);
    ca16_g2s(dst + 16u, src + 1);
  }
  ca_commit();
}

// Cut the pass starting at row li0 of the span in buffer pb: at most 32
// rows, 512 slots and kDonCap staged donor genes. Writes dbase[b].
__device__ int cut_pass(PassSmem& w, int b, int pb, int li0, int rows, int eval_only, int lane) {
  const int D4 = inst_of(w, pb).g.D4;
  const int navail = min(min(rows - li0, 32), kPassSlots / D4);
  int staged = 0;
  if (!eval_only && lane < navail) {
    const int L = w.plan[pb][li0 + lane].L;
    staged = (L <= kDonRowCap) ? L : 0;
  }
  int cum = staged;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, cum, o);
    if (lane >= o) cum += v;
  }
  const int n = __popc(__ballot_sync(0xFFFFFFFFu, lane < navail && cum <= kDonCap));   // a prefix
  if (lane < n) w.dbase[b][lane] = staged > 0 ? cum - staged : -1;
  __syncwarp();
  return n;
}

// Issue the loads of pass P: its slots into nx (lane l holds slots l + 32 k of
// the rows laid back to back) and its staged donor genes into don[b].
__device__ __forceinline__ void issue_pass(PassSmem& w, int b, const Pass& P, int eval_only, int lane,
                                           float4 (&nx)[kPassVec]) {
  const GenParams& p = inst_of(w, P.pb).g;
  const int D = p.D, D4 = p.D4;
  const size_t pitch = (size_t)p.pitch;
  const float* pop0 = p.pop0;
  const float* pop1 = p.pop1;
  // lane r < n holds the address of row r of the pass
  const float4* rp = reinterpret_cast<const float4*>(pop0);
  if (lane < P.n) {
    const int i = P.row0 + P.li0 + lane;
    const uint32_t si = eval_only ? (uint32_t)p.slots[(size_t)(p.st->gen & 1) * p.N + i]
                                  : (w.plan[P.pb][P.li0 + lane].slots & 0xFFu);
    rp = reinterpret_cast<const float4*>((si ? pop1 : pop0) + (size_t)i * pitch);
  }
  const int total = P.n * D4;
  const float inv = 1.0f / (float)D4;
  const unsigned long long rpu = reinterpret_cast<unsigned long long>(rp);
#pragma unroll
  for (int k = 0; k < kPassVec; ++k) {
    const int f = lane + 32 * k;
    const int r = (int)__fmul_rn((float)f + 0.5f, inv);          // f / D4, exact for f < 512, D4 <= 512
    const unsigned long long a = __shfl_sync(0xFFFFFFFFu, rpu, min(r, 31));
    nx[k] = (f < total) ? ld_stream(reinterpret_cast<const float4*>(a) + (f - r * D4))
                        : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  if (!eval_only) {
    for (int r = 0; r < P.n; ++r) {                                // uniform loop over the rows
      const int base = w.dbase[b][r];
      if (base < 0) continue;
      const RowPlan32& pl = w.plan[P.pb][P.li0 + r];
      const float* g1 = (((pl.slots >> 8) & 0xFFu) ? pop1 : pop0) + (size_t)pl.r1 * pitch;
      const float* g2 = (((pl.slots >> 16) & 0xFFu) ? pop1 : pop0) + (size_t)pl.r2 * pitch;
      const float* g3 = (((pl.slots >> 24) & 0xFFu) ? pop1 : pop0) + (size_t)pl.r3 * pitch;
      for (int t = lane; t < pl.L; t += 32) {
        int j = pl.jrand + t;
        if (j >= D) j -= D;
        ca4_g2s(smem_u32(&w.don[b][0][base + t]), g1 + j);
        ca4_g2s(smem_u32(&w.don[b][1][base + t]), g2 + j);
        ca4_g2s(smem_u32(&w.don[b][2][base + t]), g3 + j);
      }
    }
  }
  ca_commit();
}

// The loads of pass P have to land: registers into the pass buffer, and
// every cp.async of this lane (donor genes, span prefetches) complete.
__device__ __forceinline__ void land_pass(PassSmem& w, const Pass& P, int D4, int lane,
                                          const float4 (&nx)[kPassVec]) {
  const int total = P.n * D4;
#pragma unroll
  for (int k = 0; k < kPassVec; ++k) {
    const int f = lane + 32 * k;
    if (f < total) w.buf[f] = nx[k];
  }
  ca_wait_all();
  __syncwarp();
}

// Per-lane counters of the running span (group leaders only).
struct Cnt {
  unsigned long long kmin, masked;
  unsigned accepts;
};

// Process the landed pass P (donors in don[b]), G lanes per row.
template <int OBJ, int G>
__device__ __forceinline__ void process_pass(PassSmem& w, int b, const Pass& P, int eval_only, int lane, Cnt& c) {
  constexpr int R = 32 / G;                         // rows at a time = virtual lanes per lane
  constexpr int NS = ObjTraits<OBJ>::kSums;
  const GenParams& p = inst_of(w, P.pb).g;
  const int D = p.D, D4 = p.D4, N = p.N;
  const float F = p.F, lo = p.lo, hi = p.hi;
  const int gi = lane / G, gl = lane % G;
  for (int s0 = 0; s0 < P.n; s0 += R) {
    const int r = s0 + gi;
    const bool active = r < P.n;
    const int li = P.li0 + (active ? r : 0);
    const int i = P.row0 + li;
    float4* xs4 = &w.buf[(active ? r : 0) * D4];
    float* xs = reinterpret_cast<float*>(xs4);
    const RowPlan32& pl = w.plan[P.pb][li];
    if (!eval_only && active) {
      const int L = pl.L, jr = pl.jrand;
      const int base = w.dbase[b][r];
      const float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;
      if (base < 0) {
        const size_t pitch = (size_t)p.pitch;
        g1 = (((pl.slots >> 8) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r1 * pitch;
        g2 = (((pl.slots >> 16) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r2 * pitch;
        g3 = (((pl.slots >> 24) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r3 * pitch;
      }
      for (int t = gl; t < L; t += G) {
        int j = jr + t;
        if (j >= D) j -= D;
        float a1, a2, a3;
        if (base >= 0) {
          a1 = w.don[b][0][base + t];
          a2 = w.don[b][1][base + t];
          a3 = w.don[b][2][base + t];
        } else {
          a1 = __ldg(g1 + j);
          a2 = __ldg(g2 + j);
          a3 = __ldg(g3 + j);
        }
        xs[j] = clip_box(mutate(a1, a2, a3, F), lo, hi);
      }
    }
    __syncwarp();
    // fitness: virtual lane v = gl + G t sums slots v, v + 32, ... in order
    Acc s[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      s[t] = Acc{0.0f, 0.0f, 0.0f};
      if (!active) continue;
      for (int q = gl + G * t; q < D4; q += 32) {
        const float4 v = xs4[q];
        const int j0 = 4 * q;
        if constexpr (OBJ == kRosenbrock) {
          if (j0 + 4 < D) {
            const float nb = xs[j0 + 4];
            accum_pair(s[t], v.x, v.y);
            accum_pair(s[t], v.y, v.z);
            accum_pair(s[t], v.z, v.w);
            accum_pair(s[t], v.w, nb);
          } else {
            if (j0 + 1 < D) accum_pair(s[t], v.x, v.y);
            if (j0 + 2 < D) accum_pair(s[t], v.y, v.z);
            if (j0 + 3 < D) accum_pair(s[t], v.z, v.w);
          }
        } else {
          accum_gene<OBJ>(s[t], v.x, j0, p);
          if (j0 + 4 <= D) {
            accum_gene<OBJ>(s[t], v.y, j0 + 1, p);
            accum_gene<OBJ>(s[t], v.z, j0 + 2, p);
            accum_gene<OBJ>(s[t], v.w, j0 + 3, p);
          } else {
            if (j0 + 1 < D) accum_gene<OBJ>(s[t], v.y, j0 + 1, p);
            if (j0 + 2 < D) accum_gene<OBJ>(s[t], v.z, j0 + 2, p);
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= G) {
        const int bb = o / G;
#pragma unroll
        for (int t = 0; t < R; ++t)
          if (!(t & bb)) {
            s[t].a += s[t | bb].a;
            if (NS > 1) s[t].b += s[t | bb].b;
            if (NS > 2) s[t].c += s[t | bb].c;
          }
      } else {
        s[0].a += __shfl_xor_sync(0xFFFFFFFFu, s[0].a, o, G);
        if (NS > 1) s[0].b += __shfl_xor_sync(0xFFFFFFFFu, s[0].b, o, G);
        if (NS > 2) s[0].c += __shfl_xor_sync(0xFFFFFFFFu, s[0].c, o, G);
      }
    }
    if (active) {
      float f = finalize_fitness<OBJ>(s[0], p);      // the same value in every lane of the group
      if (f != f) f = __int_as_float(0x7F800000);
      if (eval_only) {
        if (gl == 0) {
          p.fit[i] = f;
          const unsigned long long key = best_key_of(f, i);
          c.kmin = key < c.kmin ? key : c.kmin;
        }
      } else {
        const int si = (int)(pl.slots & 0xFFu);
        const bool acc = f < pl.fit_i;
        if (gl == 0) {
          p.slots[(size_t)(pl.gpar ^ 1) * N + i] = (uint8_t)(acc ? 1 - si : si);
          c.masked += (unsigned long long)pl.L;
          if (acc) {
            c.accepts += 1u;
            p.fit[i] = f;
            const unsigned long long key = best_key_of(f, i);
            c.kmin = key < c.kmin ? key : c.kmin;
          }
          if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
          if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
          if (p.dbg_draws) {
            int* o = p.dbg_draws + 5 * (size_t)i;
            o[0] = pl.r1; o[1] = pl.r2; o[2] = pl.r3; o[3] = pl.jrand; o[4] = pl.L;
          }
        }
        if (acc) {
          float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
          for (int q = gl; q < D4; q += G) st_stream(out + q, xs4[q]);
        }
        if (p.dbg_trial) {
          float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)i * p.pitch);
          for (int q = gl; q < D4; q += G) o[q] = xs4[q];
        }
      }
    }
    __syncwarp();
  }
}

template <int OBJ>
__device__ __forceinline__ void process_g(int G, PassSmem& w, int b, const Pass& P, int eval_only, int lane,
                                          Cnt& c) {
  switch (G) {
    case 4: process_pass<OBJ, 4>(w, b, P, eval_only, lane, c); break;
    case 8: process_pass<OBJ, 8>(w, b, P, eval_only, lane, c); break;
    case 16: process_pass<OBJ, 16>(w, b, P, eval_only, lane, c); break;
    default: process_pass<OBJ, 32>(w, b, P, eval_only, lane, c); break;
  }
}

__device__ __forceinline__ void process_any(PassSmem& w, int b, const Pass& P, int eval_only, int lane, Cnt& c) {
  const BatchInst& I = inst_of(w, P.pb);
  const int G = I.lanes;                            // lanes per row of the processing
  switch (I.obj) {
    case kSphere: process_g<kSphere>(G, w, b, P, eval_only, lane, c); break;
    case kRastrigin: process_g<kRastrigin>(G, w, b, P, eval_only, lane, c); break;
    case kAckley: process_g<kAckley>(G, w, b, P, eval_only, lane, c); break;
    case kRosenbrock: process_g<kRosenbrock>(G, w, b, P, eval_only, lane, c); break;
    case kGriewank: process_g<kGriewank>(G, w, b, P, eval_only, lane, c); break;
    default: process_g<kElliptic>(G, w, b, P, eval_only, lane, c); break;
  }
}

// The span's counters go to its instance state.
__device__ __forceinline__ void flush(const GenParams& p, Cnt& c, int eval_only) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ko = __shfl_xor_sync(0xFFFFFFFFu, c.kmin, o);
    c.kmin = ko < c.kmin ? ko : c.kmin;
    c.masked += __shfl_xor_sync(0xFFFFFFFFu, c.masked, o);
    c.accepts += __shfl_xor_sync(0xFFFFFFFFu, c.accepts, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c.kmin != ~0ull) atomicMin(&p.st->best_key, c.kmin);
    if (!eval_only) {
      if (c.accepts) atomicAdd(&p.st->accepts, (unsigned long long)c.accepts);
      atomicAdd(&p.st->masked, c.masked);
    }
  }
  c.kmin = ~0ull;
  c.masked = 0ull;
  c.accepts = 0u;
}

// ctr[0]: next span to take; ctr[1]: warps finished (the last one resets both).
// FUSED (a whole generation in one cooperative launch, every instance on this
// kernel): the plans of every row first (plan tiles of 256 rows, the NEC
// table staged in the CTA's shared memory), a grid barrier (ctr[2], ctr[3]),
// the rows, and the last warp to finish closes every instance.
// A CTA whose barrier wait gives up (wait_ns) records DE_ETIMEOUT and takes
// no spans. The generation is still whole: every CTA writes its plans before
// it arrives, so the CTAs released by the barrier (the last to arrive always
// is) see every plan and take every span from the queue between them, and by
// the time the last warp finishes every CTA has arrived, so it closes the
// generation whatever its own CTA's wait did.
template <bool FUSED>
__global__ void __launch_bounds__(kPwThreads, 3)
batch_stage_kernel(const BatchInst* __restrict__ insts, const BatchSpan* __restrict__ spans, int nspans,
                   RowPlan32* __restrict__ plans, unsigned* ctr, int eval_only, const BatchTile* __restrict__ ptiles,
                   int nptiles, DevState* states, int n_inst, unsigned long long wait_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PassSmem& w = reinterpret_cast<PassSmem*>(smem_raw)[warp];
  Cnt c{~0ull, 0ull, 0u};
  float4 nx[kPassVec];
  bool go = true;
  if constexpr (FUSED) {
    // the pass buffers are free until the rows: the NEC tables go there
    static_assert(kBatchThreadsHost == 2 * kPwThreads, "two plan rows per thread");
    plan_phase<kPwThreads>(insts, ptiles, nptiles, plans, reinterpret_cast<uint32_t*>(smem_raw));
    go = grid_barrier(&ctr[2], &ctr[3], gridDim.x, wait_ns);
    if (!go && threadIdx.x == 0) atomicExch(&states[0].error, 4u);   // DE_ETIMEOUT
  }

  // span s lives in span buffer s % 3: the current one, the next one (its
  // copies in flight, desc ns) and, being located, the one after (desc nd)
  unsigned q = 0u;
  if (lane == 0 && go) q = atomicAdd(&ctr[0], 1u);
  q = __shfl_sync(0xFFFFFFFFu, q, 0);
  if (go && q < (unsigned)nspans) {
    const BatchSpan cs = spans[q];
    prefetch_span(w, 0, cs, insts, plans, eval_only, lane);
    unsigned q1 = 0u;
    if (lane == 0) q1 = atomicAdd(&ctr[0], 1u);
    q1 = __shfl_sync(0xFFFFFFFFu, q1, 0);
    BatchSpan ns;
    ns.rows = 0;
    if (q1 < (unsigned)nspans) {
      ns = spans[q1];
      prefetch_span(w, 1, ns, insts, plans, eval_only, lane);
    }
    unsigned qa = 0u;
    if (lane == 0 && ns.rows > 0) qa = atomicAdd(&ctr[0], 1u);
    qa = __shfl_sync(0xFFFFFFFFu, qa, 0);
    BatchSpan nd;
    nd.rows = 0;
    if (ns.rows > 0 && qa < (unsigned)nspans) nd = spans[qa];
    unsigned qb = 0u;
    if (lane == 0 && nd.rows > 0) qb = atomicAdd(&ctr[0], 1u);
    ca_wait_all();
    __syncwarp();

    int pb = 0, rows = cs.rows, row0 = cs.row0;
    int b = 0;
    Pass P{pb, row0, 0, 0, 0};
    P.n = cut_pass(w, b, pb, 0, rows, eval_only, lane);
    P.last = (P.n >= rows);
    int pos = P.n;
    issue_pass(w, b, P, eval_only, lane, nx);
    for (;;) {
      land_pass(w, P, inst_of(w, P.pb).g.D4, lane, nx);
      // the next pass: more rows of this span, or the first rows of the next span
      Pass Q{0, 0, 0, 0, 0};
      bool have = false;
      if (pos < rows) {
        Q.pb = pb;
        Q.row0 = row0;
        Q.li0 = pos;
        have = true;
      } else if (ns.rows > 0) {
        pb = (pb == 2) ? 0 : pb + 1;                 // its copies landed with land_pass
        rows = ns.rows;
        row0 = ns.row0;
        pos = 0;
        Q.pb = pb;
        Q.row0 = row0;
        Q.li0 = 0;
        have = true;
        ns = nd;                                     // located one span ago
        if (ns.rows > 0) prefetch_span(w, (pb == 2) ? 0 : pb + 1, ns, insts, plans, eval_only, lane);
        nd.rows = 0;
        const unsigned qn = __shfl_sync(0xFFFFFFFFu, qb, 0);
        if (ns.rows > 0 && qn < (unsigned)nspans) nd = spans[qn];
        if (lane == 0 && nd.rows > 0) qb = atomicAdd(&ctr[0], 1u);
      }
      if (have) {
        Q.n = cut_pass(w, b ^ 1, Q.pb, Q.li0, rows, eval_only, lane);
        pos = Q.li0 + Q.n;
        Q.last = (pos >= rows);
        issue_pass(w, b ^ 1, Q, eval_only, lane, nx);
      }
      process_any(w, b, P, eval_only, lane, c);
      if (P.last) flush(inst_of(w, P.pb).g, c, eval_only);
      if (!have) break;
      P = Q;
      b ^= 1;
    }
  }
  ca_wait_all();
  unsigned done = 0u;
  if (lane == 0) {
    __threadfence();
    done = atomicAdd(&ctr[1], 1u);
  }
  done = __shfl_sync(0xFFFFFFFFu, done, 0);
  if (done == gridDim.x * kPwWarps - 1u) {           // the last warp of the launch
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

}  // namespace

size_t batch_stage_smem() { return (size_t)kPwWarps * sizeof(PassSmem); }
static_assert(kBatchTableCap * 4 <= kPwWarps * (int)sizeof(PassSmem), "NEC table fits the CTA's shared memory");

// resident CTAs per SM of the two instantiations (set by prepare_batch_stage,
// the same value on every call for one device type)
static int g_stage_ctas_per_sm = 2;
static int g_fused_ctas_per_sm = 0;

cudaError_t prepare_batch_stage() {
  cudaError_t e = cudaFuncSetAttribute(batch_stage_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_stage_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_stage_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_stage_smem());
  int n = 0, m = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_kernel<false>, kPwThreads, batch_stage_smem());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, batch_stage_kernel<true>, kPwThreads, batch_stage_smem());
  if (e == cudaSuccess && n > 0) g_stage_ctas_per_sm = n;
  if (e == cudaSuccess) g_fused_ctas_per_sm = m;
  return e;
}

// grid: the row kernels' grid of two CTAs per SM; this kernel fills every SM
// with as many CTAs as fit.
cudaError_t launch_batch_stage(const BatchInst* insts, const BatchSpan* spans, int nspans, const RowPlan32* plans,
                               unsigned* ctr, int eval_only, int grid, cudaStream_t s) {
  const int g = std::max(1, grid / 2) * g_stage_ctas_per_sm;
  batch_stage_kernel<false><<<g, kPwThreads, batch_stage_smem(), s>>>(
      insts, spans, nspans, const_cast<RowPlan32*>(plans), ctr, eval_only, nullptr, 0, nullptr, 0, 0ull);
  return cudaGetLastError();
}

bool batch_fused_supported() { return g_fused_ctas_per_sm > 0; }

// One generation of every instance in one cooperative launch (all instances
// on the staged kernel): plans, rows, close. ctr: 4 counters (queue, done,
// barrier arrivals, barrier sense).
cudaError_t launch_batch_fused(const BatchInst* insts, const BatchSpan* spans, int nspans, const BatchTile* ptiles,
                               int nptiles, RowPlan32* plans, DevState* states, int n_inst, unsigned* ctr, int grid,
                               unsigned long long wait_ns, cudaStream_t s) {
  if (g_fused_ctas_per_sm <= 0) return cudaErrorNotSupported;
  if (wait_ns == 0ull) wait_ns = kWaitLimitNs;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(std::max(1, grid / 2) * g_fused_ctas_per_sm));
  cfg.blockDim = dim3(kPwThreads);
  cfg.dynamicSmemBytes = batch_stage_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_stage_kernel<true>, insts, spans, nspans, plans, ctr, 0, ptiles, nptiles,
                            states, n_inst, wait_ns);
}

}  // namespace de
