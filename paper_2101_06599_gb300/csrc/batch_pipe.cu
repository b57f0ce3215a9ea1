// batch_pipe.cu — pipelined generation of the batched instances whose rows
// are long enough to fill a warp (D >= 4 * kBpMinD4) and short enough for a
// stage (D <= 4 * kBpMaxD4), with the segment crossovers (classic
// exponential, Alg. 8; NEC, Eq. 9 + Alg. 9/10).
//
// Persistent, one CTA per SM: one producer warp and kBpCW consumer warps,
// each consumer warp with its own ring of kBpStages shared-memory stages
// (mbarrier full/empty pairs). CTA b takes rows b, b + G, b + 2G, ... of the
// row list (instance-major); its n-th row goes to consumer warp n % kBpCW.
//
// Producer: its lanes read the plans of 32 upcoming rows (donors, j_rand, L,
// slot bytes, parent fitness, written by batch_plan_kernel); lane 0 arms each
// row's stage with the expected byte count and issues the bulk copies
// (cp.async.bulk): the whole parent row and, of each donor, the 16-byte
// aligned span covering the L masked genes (two pieces when the segment
// wraps; segments longer than the span buffer read their donor genes from
// global memory). Consumer warp: patches the masked genes in shared memory
// (Eq. 1 + clipping), evaluates the trial from shared memory with its
// instance's objective, reduces over the warp, selects (strict '<'), stores
// an accepted row to the other slot buffer and releases the stage. Counters
// go to the instance's state when the warp moves to another instance.
// batch_close_kernel closes the generation afterwards. Every wait is bounded
// (ptx.cuh): a timeout records DE_ETIMEOUT in instance 0's state and stops.
#include "draws.cuh"
#include "internal.h"
#include "objectives.cuh"
#include "ptx.cuh"

namespace de {

constexpr int kBpCW = 8;           // consumer warps per CTA
constexpr int kBpStages = 2;       // stages per consumer warp
constexpr unsigned kBpErrTimeout = 4u;

struct BpMeta {
  const float* dsrc[3];            // donor rows in global memory (used when the span did not fit)
  int inst, i, jrand, L, si, r1, r2, r3, seg_ok, a0, len0;
  float fit_i;
};

struct BpPlan {
  int inst, i;
  RowPlan32 pl;
};

struct BpLayout {
  unsigned bars, abort, meta, plan, stage, total;
};

__host__ __device__ inline unsigned bp_align128(unsigned x) { return (x + 127u) & ~127u; }

__host__ __device__ inline BpLayout bp_layout(int stage_floats) {
  constexpr int slots = kBpCW * kBpStages;
  BpLayout L;
  L.bars = 0;
  L.abort = 16u * slots;
  L.meta = bp_align128(L.abort + 16u);
  L.plan = bp_align128(L.meta + (unsigned)(slots * sizeof(BpMeta)));
  L.stage = bp_align128(L.plan + (unsigned)(32 * sizeof(BpPlan)));
  L.total = L.stage + (unsigned)slots * (unsigned)stage_floats * 4u;
  return L;
}

// Partial sums of the trial held in shared memory (row), this lane's slots.
template <int OBJ>
__device__ __forceinline__ void bp_accum(const GenParams& p, const float* row, int lane, Acc& a) {
  for (int q = lane; q < p.D4; q += 32) {
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
}

template <int OBJ>
__device__ __forceinline__ float bp_fitness(const GenParams& p, const float* row, int lane) {
  Acc a{0.0f, 0.0f, 0.0f};
  bp_accum<OBJ>(p, row, lane, a);
  constexpr int NS = ObjTraits<OBJ>::kSums;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.a += __shfl_xor_sync(0xFFFFFFFFu, a.a, o);
    if (NS > 1) a.b += __shfl_xor_sync(0xFFFFFFFFu, a.b, o);
    if (NS > 2) a.c += __shfl_xor_sync(0xFFFFFFFFu, a.c, o);
  }
  float f = finalize_fitness<OBJ>(a, p);
  if (f != f) f = __int_as_float(0x7F800000);       // NaN counts as +inf
  return f;
}

__device__ __noinline__ float bp_row_fitness(int obj, const GenParams& p, const float* row, int lane) {
  switch (obj) {
    case kSphere: return bp_fitness<kSphere>(p, row, lane);
    case kRastrigin: return bp_fitness<kRastrigin>(p, row, lane);
    case kAckley: return bp_fitness<kAckley>(p, row, lane);
    case kRosenbrock: return bp_fitness<kRosenbrock>(p, row, lane);
    case kGriewank: return bp_fitness<kGriewank>(p, row, lane);
    default: return bp_fitness<kElliptic>(p, row, lane);
  }
}

__device__ __forceinline__ void bp_flag_error(const BatchInst* insts, volatile int* abort_flag) {
  atomicExch(&insts[0].g.st->error, kBpErrTimeout);
  *abort_flag = 1;
}

// Counters of one consumer warp, flushed to an instance's state.
struct BpCounters {
  int inst;
  unsigned long long masked, accepts, key;
};

__device__ __forceinline__ void bp_flush(const BatchInst* insts, BpCounters& c) {
  if (c.inst < 0) return;
  DevState* st = insts[c.inst].g.st;
  if (c.masked) atomicAdd(&st->masked, c.masked);
  if (c.accepts) atomicAdd(&st->accepts, c.accepts);
  if (c.key != ~0ull) atomicMin(&st->best_key, c.key);
  c.masked = 0;
  c.accepts = 0;
  c.key = ~0ull;
}

__global__ void __launch_bounds__(32 + 32 * kBpCW, 1)
batch_pipe_kernel(const BatchInst* __restrict__ insts, const BatchRow* __restrict__ rows, int nrows,
                  const RowPlan32* __restrict__ plans, int segcap, int stage_floats) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int SL = kBpCW * kBpStages;
  const BpLayout lay = bp_layout(stage_floats);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
  uint64_t* empty = full + SL;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + lay.abort);
  BpMeta* meta = reinterpret_cast<BpMeta*>(smem + lay.meta);
  BpPlan* plan = reinterpret_cast<BpPlan*>(smem + lay.plan);
  float* stages = reinterpret_cast<float*>(smem + lay.stage);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int ncta = (b < nrows) ? (nrows - b + G - 1) / G : 0;
  const int seg_off = stage_floats - 3 * segcap;     // floats from stage start to donor span 0

  if (threadIdx.x == 0) {
    for (int s = 0; s < SL; ++s) {
      mbar_init(smem_u32(full + s), 1u);
      mbar_init(smem_u32(empty + s), 1u);
    }
    *abort_flag = 0;
  }
  fence_mbar_init();
  __syncthreads();

  if (warp == 0) {
    // ------------------------------ producer ------------------------------
    int issued = 0;
    for (int base = 0; base < ncta; base += 32) {
      if (__shfl_sync(0xFFFFFFFFu, lane == 0 ? *abort_flag : 0, 0)) break;
      const int n = base + lane;
      if (n < ncta) {
        const BatchRow r = rows[b + n * G];
        BpPlan e;
        e.inst = r.inst;
        e.i = r.i;
        e.pl = plans[insts[r.inst].row_base + r.i];
        plan[lane] = e;
      }
      __syncwarp();
      if (lane == 0) {
        const int cnt = min(32, ncta - base);
        for (int k = 0; k < cnt; ++k) {
          const int n2 = base + k;
          const int w = n2 % kBpCW, kk = n2 / kBpCW, s = kk % kBpStages, use = kk / kBpStages;
          const int slot = w * kBpStages + s;
          if (use > 0 && !mbar_wait(smem_u32(empty + slot), (uint32_t)((use - 1) & 1))) {
            bp_flag_error(insts, abort_flag);
            break;
          }
          const BpPlan e = plan[k];
          const GenParams& p = insts[e.inst].g;
          const RowPlan32& pl = e.pl;
          const int si = (int)(pl.slots & 0xFFu);
          const int e0 = min(pl.jrand + pl.L, p.D);           // piece 0 genes [jrand, e0)
          const int a0 = pl.jrand & ~3;
          const int len0 = ((e0 + 3) & ~3) - a0;
          const int wrap = pl.jrand + pl.L - p.D;             // piece 1 genes [0, wrap)
          const int len1 = wrap > 0 ? ((wrap + 3) & ~3) : 0;
          const int seg_ok = (len0 + len1 <= segcap) ? 1 : 0;
          const float* src[4] = {(si ? p.pop1 : p.pop0) + (size_t)e.i * p.pitch,
                                 (((pl.slots >> 8) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r1 * p.pitch,
                                 (((pl.slots >> 16) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r2 * p.pitch,
                                 (((pl.slots >> 24) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl.r3 * p.pitch};
          BpMeta& m = meta[slot];
          m.dsrc[0] = src[1]; m.dsrc[1] = src[2]; m.dsrc[2] = src[3];
          m.inst = e.inst; m.i = e.i; m.jrand = pl.jrand; m.L = pl.L; m.si = si;
          m.r1 = pl.r1; m.r2 = pl.r2; m.r3 = pl.r3; m.seg_ok = seg_ok;
          m.a0 = a0; m.len0 = len0; m.fit_i = pl.fit_i;
          const uint32_t row_bytes = 16u * (uint32_t)p.D4;
          const uint32_t fb = smem_u32(full + slot);
          mbar_arrive_expect_tx(fb, row_bytes + (seg_ok ? 12u * (uint32_t)(len0 + len1) : 0u));
          float* st = stages + (size_t)slot * stage_floats;
          bulk_g2s(smem_u32(st), src[0], row_bytes, fb);
          if (seg_ok) {
#pragma unroll
            for (int k3 = 0; k3 < 3; ++k3) {
              const uint32_t sd = smem_u32(st + seg_off + k3 * segcap);
              bulk_g2s(sd, src[1 + k3] + a0, 4u * (uint32_t)len0, fb);
              if (len1 > 0) bulk_g2s(sd + 4u * (uint32_t)len0, src[1 + k3], 4u * (uint32_t)len1, fb);
            }
          }
          ++issued;
        }
      }
      __syncwarp();
    }
    // drain: the copies of the last armed stages must have landed before exit;
    // each slot is waited on for its last use only (an older phase of a slot
    // that was armed again would read as not completed)
    if (lane == 0)
      for (int w = 0; w < kBpCW; ++w) {
        const int rows_w = (issued > w) ? (issued - w + kBpCW - 1) / kBpCW : 0;   // rows given to warp w
        for (int kk = max(0, rows_w - kBpStages); kk < rows_w; ++kk)
          (void)mbar_wait(smem_u32(full + w * kBpStages + kk % kBpStages), (uint32_t)((kk / kBpStages) & 1));
      }
    __syncwarp();
  } else {
    // ------------------------------ consumers -----------------------------
    const int w = warp - 1;
    BpCounters cnt{-1, 0ull, 0ull, ~0ull};
    for (int kk = 0;; ++kk) {
      const int n = kk * kBpCW + w;
      if (n >= ncta) break;
      const int s = kk % kBpStages, use = kk / kBpStages, slot = w * kBpStages + s;
      const uint32_t fb = smem_u32(full + slot);
      int go = 0;
      if (lane == 0) {
        const bool ok = mbar_wait(fb, (uint32_t)(use & 1));
        if (!ok) bp_flag_error(insts, abort_flag);
        go = (ok && !*abort_flag) ? 1 : 0;
      }
      go = __shfl_sync(0xFFFFFFFFu, go, 0);
      if (!go) break;
      (void)mbar_try_wait(fb, (uint32_t)(use & 1));   // per-lane acquire of the completed phase
      const BpMeta m = meta[slot];
      const BatchInst& I = insts[m.inst];
      const GenParams& p = I.g;
      float* row = stages + (size_t)slot * stage_floats;
      const float* sg = row + seg_off;

      // masked genes: piece 0 = [jrand, min(jrand + L, D)), piece 1 = [0, jrand + L - D)
      const int e0 = min(m.jrand + m.L, p.D);
      const int wrap = m.jrand + m.L - p.D;
      bool patched = false;
      for (int j = m.jrand + lane; j < e0; j += 32) {
        patched = true;
        float a1, a2, a3;
        if (m.seg_ok) {
          const int o = j - m.a0;
          a1 = sg[o]; a2 = sg[segcap + o]; a3 = sg[2 * segcap + o];
        } else {
          a1 = __ldg(m.dsrc[0] + j); a2 = __ldg(m.dsrc[1] + j); a3 = __ldg(m.dsrc[2] + j);
        }
        row[j] = clip_box(mutate(a1, a2, a3, p.F), p.lo, p.hi);
      }
      for (int j = lane; j < wrap; j += 32) {
        patched = true;
        float a1, a2, a3;
        if (m.seg_ok) {
          const int o = m.len0 + j;
          a1 = sg[o]; a2 = sg[segcap + o]; a3 = sg[2 * segcap + o];
        } else {
          a1 = __ldg(m.dsrc[0] + j); a2 = __ldg(m.dsrc[1] + j); a3 = __ldg(m.dsrc[2] + j);
        }
        row[j] = clip_box(mutate(a1, a2, a3, p.F), p.lo, p.hi);
      }
      if (patched) fence_proxy_async_smem();           // patches precede the stage's next bulk fill
      __syncwarp();                                    // patched genes visible to the warp

      const float f = bp_row_fitness(I.obj, p, row, lane);
      const bool acc = f < m.fit_i;
      if (acc) {
        float4* out = reinterpret_cast<float4*>((m.si ? p.pop0 : p.pop1) + (size_t)m.i * p.pitch);
        for (int q = lane; q < p.D4; q += 32) st_stream(out + q, ld_shared_v4(row + 4 * q));
      }
      if (p.dbg_trial) {
        float4* o = reinterpret_cast<float4*>(p.dbg_trial + (size_t)m.i * p.pitch);
        for (int q = lane; q < p.D4; q += 32) o[q] = ld_shared_v4(row + 4 * q);
      }
      if (lane == 0) {
        const long long gen = p.st->gen;
        p.slots[(size_t)((gen + 1) & 1) * p.N + m.i] = (uint8_t)(acc ? 1 - m.si : m.si);
        if (acc) p.fit[m.i] = f;
        if (m.inst != cnt.inst) {
          bp_flush(insts, cnt);
          cnt.inst = m.inst;
        }
        cnt.masked += (unsigned long long)m.L;
        if (acc) {
          ++cnt.accepts;
          const unsigned long long key = best_key_of(f, m.i);
          cnt.key = key < cnt.key ? key : cnt.key;
        }
        if (p.dbg_ftrial) p.dbg_ftrial[m.i] = f;
        if (p.dbg_accept) p.dbg_accept[m.i] = (uint8_t)acc;
        if (p.dbg_draws) {
          int* o = p.dbg_draws + 5 * (size_t)m.i;
          o[0] = m.r1; o[1] = m.r2; o[2] = m.r3; o[3] = m.jrand; o[4] = m.L;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(empty + slot));
    }
    if (lane == 0) bp_flush(insts, cnt);
  }
}

unsigned batch_pipe_smem_bytes(int stage_floats) { return bp_layout(stage_floats).total; }

cudaError_t prepare_batch_pipe(size_t smem) {
  return cudaFuncSetAttribute(batch_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_batch_pipe(const BatchInst* insts, const BatchRow* rows, int nrows, const RowPlan32* plans,
                              int segcap, int stage_floats, size_t smem, int grid, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  batch_pipe_kernel<<<grid, 32 + 32 * kBpCW, smem, s>>>(insts, rows, nrows, plans, segcap, stage_floats);
  return cudaGetLastError();
}

}  // namespace de
