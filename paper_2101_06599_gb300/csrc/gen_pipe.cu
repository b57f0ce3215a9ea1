// gen_pipe.cu — instantiations and host launchers of the pipelined
// generation kernel (classic exponential and NEC crossovers).
#include "gen_pipe.cuh"
#include "internal.h"

namespace de {

template <int XO, int OBJ>
static cudaError_t pipe_one(bool prepare, const PipeParams& pp, int grid, int block, size_t smem,
                            cudaStream_t s) {
  if (prepare)
    return cudaFuncSetAttribute(gen_pipe_kernel<XO, OBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  gen_pipe_kernel<XO, OBJ><<<grid, block, smem, s>>>(pp);
  return cudaGetLastError();
}

template <int XO>
static cudaError_t pipe_xo(bool prepare, int obj, const PipeParams& pp, int grid, int block, size_t smem,
                           cudaStream_t s) {
  switch (obj) {
    case kSphere: return pipe_one<XO, kSphere>(prepare, pp, grid, block, smem, s);
    case kRastrigin: return pipe_one<XO, kRastrigin>(prepare, pp, grid, block, smem, s);
    case kAckley: return pipe_one<XO, kAckley>(prepare, pp, grid, block, smem, s);
    case kRosenbrock: return pipe_one<XO, kRosenbrock>(prepare, pp, grid, block, smem, s);
    case kGriewank: return pipe_one<XO, kGriewank>(prepare, pp, grid, block, smem, s);
    case kElliptic: return pipe_one<XO, kElliptic>(prepare, pp, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t pipe_dispatch(bool prepare, int xo, int obj, const PipeParams& pp, int grid, int block,
                                 size_t smem, cudaStream_t s) {
  if (xo == kExp) return pipe_xo<kExp>(prepare, obj, pp, grid, block, smem, s);
  if (xo == kNec) return pipe_xo<kNec>(prepare, obj, pp, grid, block, smem, s);
  return cudaErrorInvalidValue;
}

cudaError_t prepare_gen_pipe(int xo, int obj, size_t smem) {
  PipeParams pp{};
  return pipe_dispatch(true, xo, obj, pp, 0, 0, smem, nullptr);
}

cudaError_t launch_gen_pipe(int xo, int obj, const PipeParams& pp, int grid, int block, size_t smem,
                            cudaStream_t s) {
  return pipe_dispatch(false, xo, obj, pp, grid, block, smem, s);
}

unsigned pipe_smem_bytes(int S, int tcap, int stage_floats) {
  return pipe_layout(S, tcap, stage_floats).total;
}

}  // namespace de
