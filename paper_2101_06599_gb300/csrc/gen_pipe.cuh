// gen_pipe.cuh — persistent, warp-specialised generation kernel for the
// segment crossovers (classic exponential, Alg. 8; NEC, Eq. 9 + Alg. 9/10)
// at large D.
//
// Grid = one or two CTAs per SM; CTA b owns rows b, b + G, b + 2G, ... Each CTA has
// one producer warp and NC consumer threads, and a ring of S shared-memory
// stages. A stage holds one parent row and the masked segments of its three
// donor rows, filled by bulk TMA copies (cp.async.bulk) that complete on the
// stage's `full` mbarrier; consumers release it on its `empty` mbarrier.
//
// Producer warp: each lane computes the draws of one upcoming row (donors,
// j_rand, L — NEC by the threshold table held in shared memory, exp by the
// sequential walk), its slot bytes and its parent fitness, 32 rows at a
// time; lane 0 then arms each stage (expected bytes) and issues the copies:
// the whole parent row and, of each donor, only the aligned span covering
// the L masked genes (one or two pieces when the segment wraps). With S - 1
// stages in flight per SM the HBM queue stays full while consumers compute.
//
// Consumers: patch the masked genes in shared memory (Eq. 1 + clipping,
// reading the donor spans), evaluate the trial from shared memory, reduce
// (shuffles + one named barrier), decide (strict '<'), and store accepted
// rows to the other slot buffer. Counters are kept per CTA and published
// once; the last CTA to finish closes the generation. Every wait is bounded
// (ptx.cuh): on a timeout the kernel records DE_ETIMEOUT and stops.
#pragma once
#include "draws.cuh"
#include "gen_kernel.cuh"
#include "objectives.cuh"
#include "ptx.cuh"

namespace de {

constexpr int kPipeMaxStages = 8;
constexpr int kPipeMaxConsumerWarps = 16;
constexpr int kPipeTableCap = 4096;        // NEC thresholds held in shared memory
constexpr uint32_t kBulkChunk = 16384;     // bytes per bulk copy instruction
constexpr unsigned kErrTimeout = 4u;       // DE_ETIMEOUT

struct PipeParams {
  GenParams g;
  int stages;        // S
  int segcap;        // floats per donor span buffer (multiple of 4)
  int tcap;          // thresholds copied to shared memory (nT when it fits, else 0)
  int row_floats;    // 4 * D4: floats copied per parent row
  int stage_floats;  // row_floats + 3 * segcap, rounded up to 32 floats
};

struct StageMeta {
  const float* dsrc[3];  // donor rows in global memory (used when the span did not fit)
  int i, jrand, L, si;
  int r1, r2, r3, seg_ok;
  int a0, len0;          // piece 0: aligned first float and aligned length of the span
  float fit_i;
  int pad;
};

struct RowPlan {
  int i, r1, r2, r3, jrand, L, si, s1, s2, s3;
  float fit_i;
  int pad;
};

struct PipeLayout {
  unsigned bars, abort, go, meta, part, plan, tab, stage, total;
};

__host__ __device__ inline unsigned pipe_align128(unsigned x) { return (x + 127u) & ~127u; }

__host__ __device__ inline PipeLayout pipe_layout(int S, int tcap, int stage_floats) {
  PipeLayout L;
  L.bars = 0;
  L.abort = 16u * (unsigned)S;
  L.go = L.abort + 4u;
  L.meta = pipe_align128(L.abort + 16u);
  L.part = pipe_align128(L.meta + (unsigned)(S * sizeof(StageMeta)));
  L.plan = pipe_align128(L.part + (unsigned)(S * kPipeMaxConsumerWarps * 4 * sizeof(float)));
  L.tab = pipe_align128(L.plan + (unsigned)(32 * sizeof(RowPlan)));
  L.stage = pipe_align128(L.tab + 4u * (unsigned)tcap);
  L.total = L.stage + (unsigned)S * (unsigned)stage_floats * 4u;
  return L;
}

__device__ __forceinline__ int nec_length_tab(const GenParams& p, const uint32_t* tab, bool in_smem,
                                              uint32_t g, int i) {
  if (p.cr_mode != kCrGeneral) return p.cr_mode == kCrZero ? 1 : p.D;
  const uint32_t w = nec_word(p, g, i);
  return in_smem ? nec_length_of<true>(p, w, tab) : nec_length_of<false>(p, w, p.nec_tm1);
}

__device__ __forceinline__ void pipe_flag_error(const GenParams& p, volatile int* abort_flag) {
  atomicExch(&p.st->error, kErrTimeout);
  *abort_flag = 1;
}

template <int XO, int OBJ>
__global__ void __launch_bounds__(32 + 32 * kPipeMaxConsumerWarps, 1)
gen_pipe_kernel(const __grid_constant__ PipeParams pp) {
  extern __shared__ __align__(128) unsigned char smem[];
  const GenParams& p = pp.g;
  const int S = pp.stages;
  const PipeLayout lay = pipe_layout(S, pp.tcap, pp.stage_floats);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + lay.abort);  // any role may set
  volatile int* cons_go = reinterpret_cast<volatile int*>(smem + lay.go);        // consumer 0 only
  StageMeta* meta = reinterpret_cast<StageMeta*>(smem + lay.meta);
  float* part = reinterpret_cast<float*>(smem + lay.part);
  RowPlan* plan = reinterpret_cast<RowPlan*>(smem + lay.plan);
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + lay.tab);
  float* stages = reinterpret_cast<float*>(smem + lay.stage);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NC = blockDim.x - 32;             // consumer threads
  const int NCW = NC >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const int nrows = (b < p.N) ? (p.N - b + G - 1) / G : 0;
  const long long gen = p.st->gen;
  const uint32_t g = (uint32_t)gen;
  const uint8_t* slot_in = p.slots + (size_t)(gen & 1) * p.N;
  uint8_t* slot_out = p.slots + (size_t)((gen + 1) & 1) * p.N;
  const int row_bytes = pp.row_floats * 4;
  const int seg_off = pp.row_floats;          // floats from stage start to donor span 0

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(full + s), 1u);
      mbar_init(smem_u32(empty + s), (uint32_t)NCW);
    }
    *abort_flag = 0;
  }
  for (int k = threadIdx.x; k < pp.tcap; k += blockDim.x) tab[k] = p.nec_tm1[k];
  fence_mbar_init();
  __syncthreads();

  unsigned long long c_acc = 0ull, c_masked = 0ull;

  if (warp == 0) {
    // ------------------------------ producer ------------------------------
    const bool tab_smem = p.nT <= pp.tcap;
    int issued = 0;
    for (int base = 0; base < nrows; base += 32) {
      // one lane reads the flag so that the whole warp leaves together
      if (__shfl_sync(0xFFFFFFFFu, lane == 0 ? *abort_flag : 0, 0)) break;
      const int n = base + lane;
      if (n < nrows) {
        const int i = b + n * G;
        RowDraws d;
        draw_donors(p, g, i, d);
        RowPlan pl;
        pl.i = i;
        pl.r1 = d.r1; pl.r2 = d.r2; pl.r3 = d.r3; pl.jrand = d.jrand;
        if constexpr (XO == kNec) pl.L = nec_length_tab(p, tab, tab_smem, g, i);
        else pl.L = exp_walk_length(p, g, i);
        pl.si = slot_in[i];
        pl.s1 = slot_in[d.r1];
        pl.s2 = slot_in[d.r2];
        pl.s3 = slot_in[d.r3];
        pl.fit_i = p.fit[i];
        pl.pad = 0;
        plan[lane] = pl;
      }
      __syncwarp();
      if (lane == 0) {
        const int cnt = min(32, nrows - base);
        for (int k = 0; k < cnt; ++k) {
          const int n2 = base + k, s = n2 % S, use = n2 / S;
          if (use > 0 && !mbar_wait(smem_u32(empty + s), (uint32_t)((use - 1) & 1))) {
            pipe_flag_error(p, abort_flag);
            break;
          }
          const RowPlan pl = plan[k];
          const int e0 = min(pl.jrand + pl.L, p.D);           // piece 0 genes [jrand, e0)
          const int a0 = pl.jrand & ~3;
          const int len0 = ((e0 + 3) & ~3) - a0;
          const int wrap = pl.jrand + pl.L - p.D;             // piece 1 genes [0, wrap)
          const int len1 = wrap > 0 ? ((wrap + 3) & ~3) : 0;
          const int seg_ok = (len0 + len1 <= pp.segcap) ? 1 : 0;
          StageMeta& m = meta[s];
          const float* rows[4] = {(pl.si ? p.pop1 : p.pop0) + (size_t)pl.i * p.pitch,
                                  (pl.s1 ? p.pop1 : p.pop0) + (size_t)pl.r1 * p.pitch,
                                  (pl.s2 ? p.pop1 : p.pop0) + (size_t)pl.r2 * p.pitch,
                                  (pl.s3 ? p.pop1 : p.pop0) + (size_t)pl.r3 * p.pitch};
          m.dsrc[0] = rows[1]; m.dsrc[1] = rows[2]; m.dsrc[2] = rows[3];
          m.i = pl.i; m.jrand = pl.jrand; m.L = pl.L; m.si = pl.si;
          m.r1 = pl.r1; m.r2 = pl.r2; m.r3 = pl.r3; m.seg_ok = seg_ok;
          m.a0 = a0; m.len0 = len0; m.fit_i = pl.fit_i; m.pad = 0;
          const uint32_t fb = smem_u32(full + s);
          const uint32_t bytes = (uint32_t)row_bytes + (seg_ok ? 12u * (uint32_t)(len0 + len1) : 0u);
          mbar_arrive_expect_tx(fb, bytes);
          float* st = stages + (size_t)s * pp.stage_floats;
          const uint32_t dst = smem_u32(st);
          for (uint32_t off = 0; off < (uint32_t)row_bytes; off += kBulkChunk)
            bulk_g2s(dst + off, reinterpret_cast<const char*>(rows[0]) + off,
                     min(kBulkChunk, (uint32_t)row_bytes - off), fb);
          if (seg_ok) {
#pragma unroll
            for (int k3 = 0; k3 < 3; ++k3) {
              const uint32_t sd = smem_u32(st + seg_off + k3 * pp.segcap);
              bulk_g2s(sd, rows[1 + k3] + a0, 4u * (uint32_t)len0, fb);
              if (len1 > 0) bulk_g2s(sd + 4u * (uint32_t)len0, rows[1 + k3], 4u * (uint32_t)len1, fb);
            }
          }
          ++issued;
        }
      }
      __syncwarp();
    }
    // drain: the copies of the last armed stages must have landed before exit
    if (lane == 0)
      for (int n2 = max(0, issued - S); n2 < issued; ++n2)
        (void)mbar_wait(smem_u32(full + (n2 % S)), (uint32_t)((n2 / S) & 1));
    __syncwarp();
  } else {
    // ------------------------------ consumers -----------------------------
    const int ct = threadIdx.x - 32, cw = ct >> 5;
    for (int n = 0; n < nrows; ++n) {
      const int s = n % S;
      const uint32_t par = (uint32_t)((n / S) & 1);
      const uint32_t fb = smem_u32(full + s);
      // consumer 0 alone waits and decides; the others learn the outcome
      // from cons_go, which only consumer 0 writes, so all leave together
      if (ct == 0) {
        const bool ok = mbar_wait(fb, par);
        if (!ok) pipe_flag_error(p, abort_flag);
        *cons_go = (ok && !*abort_flag) ? 1 : 0;
      }
      named_bar_sync(1, NC);
      if (!*cons_go) break;
      (void)mbar_try_wait(fb, par);              // per-thread acquire of the completed phase
      const StageMeta m = meta[s];
      float* row = stages + (size_t)s * pp.stage_floats;
      const float* sg = row + seg_off;

      // 1. masked genes: piece 0 = [jrand, min(jrand + L, D)), piece 1 = [0, jrand + L - D)
      const int e0 = min(m.jrand + m.L, p.D);
      const int wrap = m.jrand + m.L - p.D;
      bool patched = false;
      for (int j = m.jrand + ct; j < e0; j += NC) {
        patched = true;
        float a1, a2, a3;
        if (m.seg_ok) {
          const int o = j - m.a0;
          a1 = sg[o]; a2 = sg[pp.segcap + o]; a3 = sg[2 * pp.segcap + o];
        } else {
          a1 = __ldg(m.dsrc[0] + j); a2 = __ldg(m.dsrc[1] + j); a3 = __ldg(m.dsrc[2] + j);
        }
        row[j] = repair_gene(mutate(a1, a2, a3, p.F), row[j], p);
      }
      for (int j = ct; j < wrap; j += NC) {
        patched = true;
        float a1, a2, a3;
        if (m.seg_ok) {
          const int o = m.len0 + j;
          a1 = sg[o]; a2 = sg[pp.segcap + o]; a3 = sg[2 * pp.segcap + o];
        } else {
          a1 = __ldg(m.dsrc[0] + j); a2 = __ldg(m.dsrc[1] + j); a3 = __ldg(m.dsrc[2] + j);
        }
        row[j] = repair_gene(mutate(a1, a2, a3, p.F), row[j], p);
      }
      if (patched) fence_proxy_async_smem();      // patches precede the stage's next bulk fill
      named_bar_sync(2, NC);                      // patched genes visible to every consumer

      // 2. fitness of the trial, from shared memory: slots whose four genes
      //    are all in the row go two at a time into two independent partial
      //    sums (shorter dependency chains), the rest through the checked loop
      Acc a{0.0f, 0.0f, 0.0f}, a2{0.0f, 0.0f, 0.0f};
      const int qfull = p.D >> 2;
      int q0 = ct;
      for (; q0 + NC < qfull; q0 += 2 * NC) {
        const float4 v0 = ld_shared_v4(row + 4 * q0);
        const float4 v1 = ld_shared_v4(row + 4 * (q0 + NC));
        const int j0 = 4 * q0, j1 = 4 * (q0 + NC);
        if constexpr (OBJ == kRosenbrock) {
          accum_pair(a, v0.x, v0.y);
          accum_pair(a2, v1.x, v1.y);
          accum_pair(a, v0.y, v0.z);
          accum_pair(a2, v1.y, v1.z);
          accum_pair(a, v0.z, v0.w);
          accum_pair(a2, v1.z, v1.w);
          if (j0 + 4 < p.D) accum_pair(a, v0.w, row[j0 + 4]);
          if (j1 + 4 < p.D) accum_pair(a2, v1.w, row[j1 + 4]);
        } else {
          accum_gene<OBJ>(a, v0.x, j0, p);
          accum_gene<OBJ>(a2, v1.x, j1, p);
          accum_gene<OBJ>(a, v0.y, j0 + 1, p);
          accum_gene<OBJ>(a2, v1.y, j1 + 1, p);
          accum_gene<OBJ>(a, v0.z, j0 + 2, p);
          accum_gene<OBJ>(a2, v1.z, j1 + 2, p);
          accum_gene<OBJ>(a, v0.w, j0 + 3, p);
          accum_gene<OBJ>(a2, v1.w, j1 + 3, p);
        }
      }
      a.a += a2.a;
      a.b += a2.b;
      a.c += a2.c;
      for (int q = q0; q < p.D4; q += NC) {
        const float4 v = ld_shared_v4(row + 4 * q);
        const int j0 = 4 * q;
        if constexpr (OBJ == kRosenbrock) {
          if (j0 + 1 < p.D) accum_pair(a, v.x, v.y);
          if (j0 + 2 < p.D) accum_pair(a, v.y, v.z);
          if (j0 + 3 < p.D) accum_pair(a, v.z, v.w);
          if (j0 + 4 < p.D) accum_pair(a, v.w, row[j0 + 4]);
        } else {
          accum_gene<OBJ>(a, v.x, j0, p);
          if (j0 + 1 < p.D) accum_gene<OBJ>(a, v.y, j0 + 1, p);
          if (j0 + 2 < p.D) accum_gene<OBJ>(a, v.z, j0 + 2, p);
          if (j0 + 3 < p.D) accum_gene<OBJ>(a, v.w, j0 + 3, p);
        }
      }
      int dummy = 0;
      warp_reduce(a, dummy, ObjTraits<OBJ>::kSums);
      float* ps = part + (size_t)s * kPipeMaxConsumerWarps * 4;
      if (lane == 0) {
        ps[4 * cw + 0] = a.a;
        ps[4 * cw + 1] = a.b;
        ps[4 * cw + 2] = a.c;
      }
      named_bar_sync(3, NC);

      // 3. every consumer forms the same row value and decision
      Acc r{0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int w = 0; w < kPipeMaxConsumerWarps; ++w) {
        if (w < NCW) {
          r.a += ps[4 * w + 0];
          r.b += ps[4 * w + 1];
          r.c += ps[4 * w + 2];
        }
      }
      float f = finalize_fitness<OBJ>(r, p);
      if (f != f) f = __int_as_float(0x7F800000);
      const bool acc = f < m.fit_i;
      if (acc) {
        float4* out = reinterpret_cast<float4*>((m.si ? p.pop0 : p.pop1) + (size_t)m.i * p.pitch);
        for (int q = ct; q < p.D4; q += NC) st_stream(out + q, ld_shared_v4(row + 4 * q));
      }
      if (p.dbg_trial) {
        float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)m.i * p.pitch);
        for (int q = ct; q < p.D4; q += NC) o[q] = ld_shared_v4(row + 4 * q);
      }
      if (ct == 0) {
        slot_out[m.i] = (uint8_t)(acc ? 1 - m.si : m.si);
        if (acc) {
          p.fit[m.i] = f;
          atomicMin(&p.st->best_key, best_key_of(f, m.i));
          ++c_acc;
        }
        c_masked += (unsigned long long)m.L;
        if (p.dbg_ftrial) p.dbg_ftrial[m.i] = f;
        if (p.dbg_accept) p.dbg_accept[m.i] = (uint8_t)acc;
        if (p.dbg_draws) {
          int* o = p.dbg_draws + 5 * (size_t)m.i;
          o[0] = m.r1; o[1] = m.r2; o[2] = m.r3; o[3] = m.jrand; o[4] = m.L;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(empty + s));
    }
  }

  __syncthreads();
  if (threadIdx.x == 32) {
    if (c_acc) atomicAdd(&p.st->accepts, c_acc);
    if (c_masked) atomicAdd(&p.st->masked, c_masked);
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

}  // namespace de
