// sr_tc.cu — tcgen05 product of the shifted-rotated objectives with a fused
// fitness epilogue: Z = A' B'^T over K' = 3D, the split operands (BF16, or
// FP16 of power-of-two-scaled values) concatenated along K as (a_lo, R_hi),
// (a_hi, R_lo), (a_hi, R_hi), FP32 accumulation in tensor memory. The two
// correction products come first: their partial sums are about 2^-8 (BF16)
// or 2^-11 (FP16) of the leading product's, so their 2D/16 accumulation
// steps add almost nothing to the accumulator's rounding, which the leading
// D/16 steps then dominate (the error bound counts it that way).
//
// One CTA per 128 x 256 output tile; 6 warps:
//   warp 0      one thread issues 2D tensor loads (TMA, 128-byte swizzle) of
//               the A and B tiles (K = 64 per stage) into a 4-stage ring
//               (full / empty mbarriers);
//   warp 1      allocates 256 TMEM columns; one thread issues
//               tcgen05.mma.cta_group::1.kind::f16 (M 128, N 256, K 16, BF16
//               or FP16 inputs, FP32 accumulator), commits each stage's MMAs to the
//               stage's empty barrier and the last to the accumulator barrier;
//               frees TMEM at the end;
//   warps 2..5  read the accumulator with tcgen05.ld (warp w reads TMEM lanes
//               32 (w mod 4) .. + 31 = its 32 tile rows), undo the operands'
//               power-of-two scaling (FP16) and reduce g(z) and w |z| over
//               the tile's 256 columns into per-row partials.
// Every mbarrier wait is bounded (1 s); on a timeout the kernel records
// DE_ETIMEOUT, lets issued copies and MMAs drain (bounded), frees TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "internal.h"
#include "ptx.cuh"
#include "sr_common.cuh"

namespace de {

constexpr int kTcBM = 128, kTcBN = 256, kTcBK = 64, kTcStages = 4, kTcThreads = 192;
constexpr uint32_t kTcStageA = kTcBM * kTcBK * 2;   // 16 KB
constexpr uint32_t kTcStageB = kTcBN * kTcBK * 2;   // 32 KB
constexpr uint32_t kTcTmemCols = 256;
constexpr size_t kTcSmem = 1024 /*alignment slack*/ + kTcStages * (kTcStageA + kTcStageB) + 256;

struct TcParams {
  SrParams sp;
  CUtensorMap ta_hi, ta_lo, tr_hi, tr_lo;
  uint32_t idesc;          // instruction descriptor (operand type)
};

// K-major, 128-byte-swizzled shared-memory matrix descriptor: start address,
// leading byte offset 1 (unused for this layout), stride byte offset 1024
// (8 rows x 128 bytes), descriptor version 1, swizzle mode 128B.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (type code 1) or
// both FP16 (type code 0), both K-major, N = 256, M = 128.
constexpr uint32_t kTcIdescF16 = (1u << 4) | ((uint32_t)(kTcBN >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
constexpr uint32_t kTcIdescBF16 = kTcIdescF16 | (1u << 7) | (1u << 10);

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1) sr_tc_kernel(const __grid_constant__ TcParams tp) {
  griddep_wait();                                  // the trial kernel has written the operands
  griddep_launch_dependents();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTcStages * kTcStageA;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kTcStages * kTcStageB);
  uint64_t* empty = full + kTcStages;
  uint64_t* accum = empty + kTcStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const SrParams& sp = tp.sp;
  const GenParams& p = sp.g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_n = blockIdx.x, tile_m = blockIdx.y;
  const int KT = p.D / kTcBK;
  const int total = 3 * KT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(full + s), 1u);
      mbar_init(smem_u32(empty + s), 1u);
    }
    mbar_init(smem_u32(accum), 1u);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int issued = 0;
    for (int it = 0; it < total; ++it) {
      const int s = it % kTcStages, use = it / kTcStages;
      if (use > 0 && !mbar_wait(smem_u32(empty + s), (uint32_t)((use - 1) & 1))) {
        atomicExch(&p.st->error, 4u);
        break;
      }
      const int seg = it / KT, kt = it - seg * KT;
      const CUtensorMap* ma = (seg == 0) ? &tp.ta_lo : &tp.ta_hi;
      const CUtensorMap* mb = (seg == 1) ? &tp.tr_lo : &tp.tr_hi;
      const uint32_t fb = smem_u32(full + s);
      mbar_arrive_expect_tx(fb, kTcStageA + kTcStageB);
      tma_load_2d(smem_u32(sA + s * kTcStageA), ma, kt * kTcBK, tile_m * kTcBM, fb);
      tma_load_2d(smem_u32(sB + s * kTcStageB), mb, kt * kTcBK, tile_n * kTcBN, fb);
      ++issued;
    }
    // copies of the last stages must have landed before the CTA can exit
    for (int it = (issued > kTcStages ? issued - kTcStages : 0); it < issued; ++it)
      (void)mbar_wait(smem_u32(full + (it % kTcStages)), (uint32_t)((it / kTcStages) & 1));
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int it = 0; it < total; ++it) {
      const int s = it % kTcStages, use = it / kTcStages;
      if (!mbar_wait(smem_u32(full + s), (uint32_t)(use & 1))) {
        atomicExch(&p.st->error, 4u);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * kTcStageA), b0 = smem_u32(sB + s * kTcStageB);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk)
        umma_f16(tmem, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32), tp.idesc,
                 (it > 0 || kk > 0) ? 1u : 0u);
      umma_commit(smem_u32(empty + s));
    }
    umma_commit(smem_u32(accum));              // after every MMA issued above has completed
  } else if (warp >= 2) {
    // ---- epilogue ----
    const bool ok = mbar_wait(smem_u32(accum), 0u);
    tc_fence_after();
    const int q = warp & 3;                    // TMEM lane quadrant of this warp
    const int m = tile_m * kTcBM + 32 * q + lane;
    float sg = 0.0f, sw = 0.0f;
    if (ok) {
      // one loop per objective (the objective is uniform): no per-value test
      auto tile_sums = [&](auto obj_tag) {
        constexpr int OBJ = decltype(obj_tag)::value;
#pragma unroll 1
        for (int c0 = 0; c0 < kTcBN; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const float z = __uint_as_float(r[c]) * sp.z_scale;   // exact: a power of two
            const float w = sr_weight(OBJ, tile_n * kTcBN + c0 + c, p.ell_k);
            sg += sr_g(OBJ, z, w);
            sw = fmaf(w, fabsf(z), sw);
          }
        }
      };
      if (sp.obj == kSrElliptic) tile_sums(std::integral_constant<int, kSrElliptic>{});
      else tile_sums(std::integral_constant<int, kSrRastrigin>{});
    } else {
      atomicExch(&p.st->error, 4u);
    }
    if (m < p.N) {
      sp.part_g[(size_t)m * sp.nct + tile_n] = sg;
      sp.part_w[(size_t)m * sp.nct + tile_n] = sw;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  }
  return fn;
}

static bool encode_half_2d(CUtensorMap* tm, const void* ptr, uint64_t inner, uint64_t outer, uint32_t box_outer,
                           bool fp16) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcBK, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr),
             dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool sr_tc_supported(int D) {
  if (D % kTcBN != 0 || D < kTcBN) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3 && tensor_map_encoder() != nullptr;
}

cudaError_t prepare_sr_tc() {
  return cudaFuncSetAttribute(sr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
}

cudaError_t launch_sr_gemm_tc(const SrParams& sp, cudaStream_t s) {
  TcParams tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.sp = sp;
  const int N = sp.g.N, D = sp.g.D;
  const bool fp16 = sp.prec == 3;
  tp.idesc = fp16 ? kTcIdescF16 : kTcIdescBF16;
  if (!encode_half_2d(&tp.ta_hi, sp.a_hi, (uint64_t)D, (uint64_t)N, kTcBM, fp16) ||
      !encode_half_2d(&tp.ta_lo, sp.a_lo, (uint64_t)D, (uint64_t)N, kTcBM, fp16) ||
      !encode_half_2d(&tp.tr_hi, sp.rot_hi, (uint64_t)D, (uint64_t)D, kTcBN, fp16) ||
      !encode_half_2d(&tp.tr_lo, sp.rot_lo, (uint64_t)D, (uint64_t)D, kTcBN, fp16))
    return cudaErrorInvalidValue;
  const dim3 grid((unsigned)(D / kTcBN), (unsigned)((N + kTcBM - 1) / kTcBM));
  return launch_pdl(sr_tc_kernel, grid, dim3(kTcThreads), kTcSmem, s, tp);
}

}  // namespace de
