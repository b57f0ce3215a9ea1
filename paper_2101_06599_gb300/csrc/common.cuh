// common.cuh — device-side data layout and small helpers shared by the
// generation, initialisation and evaluation kernels.
//
// Layout in HBM (one context):
//   pop[2]   : two N x pitch FP32 slot buffers; pitch = D rounded up to 8
//              floats so every row starts on a 32-byte sector;
//   slots    : 2 x N bytes; slots[g & 1][i] names the buffer holding row i
//              at the start of generation g, slots[(g+1) & 1][i] is written
//              during generation g (a donor read never races a row write);
//   fit      : N FP32 fitness values, read and written only by row i's CTA;
//   state    : DevState (generation counter, best key, counters);
//   nec_tm1  : NEC thresholds T_n - 1 (uint32, n = 1 .. nT), see draws.cuh.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "philox.cuh"

namespace de {

enum Xo : int { kBin = 0, kExp = 1, kNec = 2 };
enum Obj : int {
  kSphere = 0, kRastrigin = 1, kAckley = 2, kRosenbrock = 3, kGriewank = 4, kElliptic = 5,
  kSrRastrigin = 6, kSrElliptic = 7
};

// Launch shapes: at most kMaxThreads threads per row-CTA, each holding
// kVecChoices[v] float4 slots of the row.
constexpr int kMaxThreads = 512;
constexpr int kVecChoices[5] = {1, 2, 4, 8, 16};

// Cr special cases of Eq. (9).
enum CrMode : int { kCrGeneral = 0, kCrZero = 1, kCrOne = 2 };
// Base index rules (de_base in de.h).
enum BaseRule : int { kBaseDistinct = 0, kBaseRandom = 1, kBaseOffset = 2, kBasePermutation = 3, kBaseBest = 4 };

struct DevState {
  unsigned long long best_key;   // (orderable FP32 bits << 32) | row
  long long gen;                 // generations completed
  long long best_gen;            // generation of the last strict improvement
  unsigned long long accepts;    // accepted trials, cumulative
  unsigned long long masked;     // masked genes (sum L or popcount), cumulative
  unsigned long long reselected; // rows re-evaluated in FP32 (rotated path)
  unsigned int done;             // CTAs finished in the running generation
  unsigned int error;            // sticky device error code (0 = none)
  float best_f;                  // best fitness at the end of the last generation
  int base_row;                  // best row when the last generation closed (DE/best/1's base)
  float pad_[2];
  double incumbent_f64;          // shifted-rotated: FP64 objective of the best row
  long long incumbent_gen;       // generation of that re-evaluation (-1 = none)
};

struct GenParams {
  float* pop0;
  float* pop1;
  float* fit;
  uint8_t* slots;
  DevState* st;
  const uint32_t* nec_tm1;  // T_n - 1 for n = 1 .. nT (non-increasing)
  int nT;
  int N, D, pitch, D4;      // D4 = ceil(D / 4) float4 slots per row
  float F, lo, hi;
  int cr_mode;
  int base;                 // base index rule (kBaseDistinct .. kBaseBest)
  int repair;               // bound repair: 0 clip, 1 midpoint between the violated bound and the target
  unsigned long long cr_t;  // ceil(Cr * 2^32): rand < Cr  <=>  w < cr_t
  uint32_t cr_lt;           // min(cr_t, 2^32 - 1): w < cr_lt as a 32-bit test when cr_all is 0
  int cr_all;               // cr_t = 2^32: every word passes
  Key2 key;
  uint32_t inst;
  float ackley_b;
  float ell_k;              // elliptic: exponent step 6 log2(10) / (D - 1)
  float nec_k;              // 1 / -log2(Cr) for 0 < Cr < 1 (the NEC lookup's first guess), else 0
  // test hook outputs (device, may be null)
  float* dbg_trial;         // N x pitch
  float* dbg_ftrial;        // N
  uint8_t* dbg_accept;      // N
  int* dbg_draws;           // N x 5
  RoundKeys rk;             // key's Philox round keys (kernels drawing a block per few genes)
};

// Programmatic dependent launch. A kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream is still running (once
// every CTA of that kernel has called griddep_launch_dependents or exited):
// its launch overlaps the previous kernel's tail instead of following it.
// griddep_wait blocks until the previous kernel has completed and its memory
// is visible; every kernel launched this way calls it before it reads or
// writes anything. Both are no-ops for a kernel launched without it.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// FP32 -> uint32 whose unsigned order is the float order; NaN maps above +inf.
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  if (f != f) return 0xFFFFFFFFu;
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__device__ __forceinline__ unsigned long long best_key_of(float f, int row) {
  return ((unsigned long long)ordered_bits(f) << 32) | (uint32_t)row;
}

// Streaming 128-bit load through the non-coherent path, not kept in L1
// (every byte of a parent row is read once per generation).
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
// Read-only 128-bit load (donor rows: few bytes, may be reused by other rows).
__device__ __forceinline__ float4 ld_ro(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
// Streaming 128-bit store (accepted rows are not read again this generation).
__device__ __forceinline__ void st_stream(float4* p, float4 v) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

__device__ __forceinline__ float& lane_of(float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Bound repair: clip to [lo, hi] (exact).
__device__ __forceinline__ float clip_box(float v, float lo, float hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Bound repair of a mutant gene v whose target (parent) gene is x, itself in
// the box: clip to [lo, hi], or (repair = 1) the midpoint between the
// violated bound and x, fl(fl(bound + x) 0.5), which stays in the box.
__device__ __forceinline__ float midpoint_box(float v, float x, float lo, float hi) {
  if (v < lo) return __fmul_rn(__fadd_rn(lo, x), 0.5f);
  if (v > hi) return __fmul_rn(__fadd_rn(hi, x), 0.5f);
  return v;
}
__device__ __forceinline__ float repair_gene(float v, float x, const GenParams& p) {
  return p.repair ? midpoint_box(v, x, p.lo, p.hi) : clip_box(v, p.lo, p.hi);
}

// Eq. (1) for one gene, each operation rounded once: x1 + F (x2 - x3).
__device__ __forceinline__ float mutate(float x1, float x2, float x3, float F) {
  return __fadd_rn(x1, __fmul_rn(F, __fsub_rn(x2, x3)));
}

// The masked genes (bits of m) of one float4 slot v of a target row take the
// mutant x1 + F (x2 - x3) of the donor slots a1, a2, a3, repaired. The repair
// mode is tested once per slot (uniform across the launch), so clipping, the
// common case, stays two comparisons per gene.
template <int kRepair = -1>                      // 0 clip, 1 midpoint, -1 as p.repair says
__device__ __forceinline__ void mutate_slot(float4& v, const float4& a1, const float4& a2, const float4& a3,
                                            unsigned m, const GenParams& p) {
  if (kRepair == 0 || (kRepair < 0 && !p.repair)) {
    if (m & 1u) v.x = clip_box(mutate(a1.x, a2.x, a3.x, p.F), p.lo, p.hi);
    if (m & 2u) v.y = clip_box(mutate(a1.y, a2.y, a3.y, p.F), p.lo, p.hi);
    if (m & 4u) v.z = clip_box(mutate(a1.z, a2.z, a3.z, p.F), p.lo, p.hi);
    if (m & 8u) v.w = clip_box(mutate(a1.w, a2.w, a3.w, p.F), p.lo, p.hi);
  } else {
    if (m & 1u) v.x = midpoint_box(mutate(a1.x, a2.x, a3.x, p.F), v.x, p.lo, p.hi);
    if (m & 2u) v.y = midpoint_box(mutate(a1.y, a2.y, a3.y, p.F), v.y, p.lo, p.hi);
    if (m & 4u) v.z = midpoint_box(mutate(a1.z, a2.z, a3.z, p.F), v.z, p.lo, p.hi);
    if (m & 8u) v.w = midpoint_box(mutate(a1.w, a2.w, a3.w, p.F), v.w, p.lo, p.hi);
  }
}

}  // namespace de
