// batch_stream.cu — the streaming generation of the batched instances with
// rows of at least 4 * kBsMinD4 genes: one warp per row, the row walked in
// chunks (gen_stream.cuh: parent loads, crossover masks, the donor float4s of
// masked slots, mutation and clipping, partial sums), a warp reduction, the
// strict selection, and only a winning row recomputed and stored. Nothing of
// a row is held across the reduction, so the kernel runs at 64 registers and
// four CTAs per SM: 32 rows in flight per SM.
//
// The draws come from batch_plan_kernel's plans. Warp w of the grid takes the
// rows [seg[w], seg[w + 1]) of the row list (instance-major; the host cuts it
// into equal numbers of genes per warp), so a warp's rows mostly share an
// instance and its counters reach the instance's state once per instance.
// batch_close_kernel closes the generation afterwards.
#include "gen_stream.cuh"
#include "internal.h"

namespace de {

constexpr int kBsWarps = 8;

struct BsCounters {
  int inst;
  unsigned long long masked, accepts, key;
};

__device__ __forceinline__ void bs_flush(const BatchInst* insts, BsCounters& c) {
  if (c.inst < 0) return;
  DevState* st = insts[c.inst].g.st;
  if (c.masked) atomicAdd(&st->masked, c.masked);
  if (c.accepts) atomicAdd(&st->accepts, c.accepts);
  if (c.key != ~0ull) atomicMin(&st->best_key, c.key);
  c.masked = 0;
  c.accepts = 0;
  c.key = ~0ull;
}

// One row (instance inst, row i) of a warp; lane 0 updates the counters.
template <int XO, int OBJ>
__device__ __noinline__ void batch_stream_row(const BatchInst* insts, int inst, int i,
                                              const RowPlan32* __restrict__ plans, BsCounters& c) {
  const int lane = threadIdx.x & 31;
  const BatchInst& I = insts[inst];
  const GenParams& p = I.g;
  const RowPlan32* pl = plans + I.row_base + i;
  const long long gen = p.st->gen;
  const uint32_t slots = pl->slots;
  const int si = (int)(slots & 0xFFu);
  StreamRow r;
  r.x = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)i * p.pitch);
  r.d1 = reinterpret_cast<const float4*>((((slots >> 8) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl->r1 * p.pitch);
  r.d2 = reinterpret_cast<const float4*>((((slots >> 16) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl->r2 * p.pitch);
  r.d3 = reinterpret_cast<const float4*>((((slots >> 24) & 0xFFu) ? p.pop1 : p.pop0) + (size_t)pl->r3 * p.pitch);
  r.jrand = pl->jrand;
  r.L = pl->L;
  r.i = i;
  r.g = (uint32_t)gen;
  int cnt = 0;
  const float f = stream_row_value<XO, OBJ>(p, r, lane, cnt);
  const int acc = (f < pl->fit_i) ? 1 : 0;
  const int Lrow = (XO == kBin) ? cnt : r.L;
  if (lane == 0) {
    p.slots[(size_t)((gen + 1) & 1) * p.N + i] = (uint8_t)(acc ? 1 - si : si);
    if (acc) p.fit[i] = f;
    if (c.inst != inst) {
      bs_flush(insts, c);
      c.inst = inst;
    }
    c.masked += (unsigned long long)Lrow;
    if (acc) {
      ++c.accepts;
      const unsigned long long key = best_key_of(f, i);
      c.key = key < c.key ? key : c.key;
    }
    if (p.dbg_ftrial) p.dbg_ftrial[i] = f;
    if (p.dbg_accept) p.dbg_accept[i] = (uint8_t)acc;
    if (p.dbg_draws) {
      int* o = p.dbg_draws + 5 * (size_t)i;
      o[0] = pl->r1; o[1] = pl->r2; o[2] = pl->r3; o[3] = r.jrand; o[4] = Lrow;
    }
  }
  if (acc) {
    float4* out = reinterpret_cast<float4*>((si ? p.pop0 : p.pop1) + (size_t)i * p.pitch);
    stream_row_store<XO>(p, r, lane, out);
  }
}

template <int OBJ>
__device__ __forceinline__ void batch_stream_row_xo(int xo, const BatchInst* insts, int inst, int i,
                                                    const RowPlan32* plans, BsCounters& c) {
  if (xo == kBin) batch_stream_row<kBin, OBJ>(insts, inst, i, plans, c);
  else if (xo == kExp) batch_stream_row<kExp, OBJ>(insts, inst, i, plans, c);
  else batch_stream_row<kNec, OBJ>(insts, inst, i, plans, c);
}

__global__ void __launch_bounds__(kBsWarps * 32, 4)
batch_stream_kernel(const BatchInst* __restrict__ insts, const BatchRow* __restrict__ rows,
                    const int* __restrict__ seg, const RowPlan32* __restrict__ plans) {
  const int gw = blockIdx.x * kBsWarps + (threadIdx.x >> 5);
  BsCounters c{-1, 0ull, 0ull, ~0ull};
  const int k1 = seg[gw + 1];
  for (int k = seg[gw]; k < k1; ++k) {
    const BatchRow br = rows[k];
    const int obj = insts[br.inst].obj, xo = insts[br.inst].xo;   // uniform over the warp
    switch (obj) {
      case kSphere: batch_stream_row_xo<kSphere>(xo, insts, br.inst, br.i, plans, c); break;
      case kRastrigin: batch_stream_row_xo<kRastrigin>(xo, insts, br.inst, br.i, plans, c); break;
      case kAckley: batch_stream_row_xo<kAckley>(xo, insts, br.inst, br.i, plans, c); break;
      case kRosenbrock: batch_stream_row_xo<kRosenbrock>(xo, insts, br.inst, br.i, plans, c); break;
      case kGriewank: batch_stream_row_xo<kGriewank>(xo, insts, br.inst, br.i, plans, c); break;
      default: batch_stream_row_xo<kElliptic>(xo, insts, br.inst, br.i, plans, c); break;
    }
  }
  if ((threadIdx.x & 31) == 0) bs_flush(insts, c);
}

cudaError_t launch_batch_stream(const BatchInst* insts, const BatchStreamLaunch& b, const RowPlan32* plans,
                                cudaStream_t s) {
  if (b.nrows <= 0) return cudaSuccess;
  batch_stream_kernel<<<b.grid, kBsWarps * 32, 0, s>>>(insts, b.rows, b.seg, plans);
  return cudaGetLastError();
}

}  // namespace de
