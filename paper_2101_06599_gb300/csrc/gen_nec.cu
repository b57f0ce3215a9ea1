// gen_nec.cu — instantiations of the fused generation kernel for one crossover.
#include "gen_kernel.cuh"
#include "internal.h"

namespace de {

cudaError_t launch_gen_nec(int obj, int vidx, const GenParams& p, int block, cudaStream_t s) {
  return launch_gen_xo<kNec>(obj, vidx, p, block, s);
}

}  // namespace de
