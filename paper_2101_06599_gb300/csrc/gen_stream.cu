// gen_stream.cu — instantiations of the streaming (warp-per-row) generation kernel.
#include "gen_stream.cuh"
#include "internal.h"

namespace de {

// Allows the binomial instantiation its mask bytes in shared memory (once per
// context, outside any stream capture).
cudaError_t prepare_gen_stream(int xo, int obj) {
  return xo == kBin ? prepare_stream_xo<kBin>(obj) : cudaSuccess;
}

cudaError_t launch_gen_stream(int xo, int obj, const GenParams& p, cudaStream_t s) {
  if (xo == kBin) return launch_stream_xo<kBin>(obj, p, s);
  if (xo == kExp) return launch_stream_xo<kExp>(obj, p, s);
  return launch_stream_xo<kNec>(obj, p, s);
}

}  // namespace de
