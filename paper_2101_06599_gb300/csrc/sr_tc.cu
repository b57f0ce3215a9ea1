// sr_tc.cu — tcgen05 product of the shifted-rotated objectives (BF16 split
// operands, FP32 accumulation in tensor memory, fused fitness epilogue).
#include "internal.h"
#include "sr_common.cuh"

namespace de {

bool sr_tc_supported(int D) { (void)D; return false; }

cudaError_t launch_sr_gemm_tc(const SrParams& sp, cudaStream_t s) {
  (void)sp; (void)s;
  return cudaErrorNotSupported;
}

}  // namespace de
