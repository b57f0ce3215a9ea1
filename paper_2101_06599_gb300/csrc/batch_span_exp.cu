// batch_span_exp.cu — the span row kernel (batch_span.cuh) instantiated for
// one crossover, in its own translation unit so the three compile in parallel.
#include "batch_span.cuh"

namespace de {

cudaError_t launch_batch_span_exp(const BatchInst* insts, const BatchSpan* spans, int nspans, const RowPlan32* plans,
                                unsigned* ctr, int eval_only, int grid, cudaStream_t s) {
  return launch_batch_span_xo<kExp>(insts, spans, nspans, plans, ctr, eval_only, grid, s);
}

}  // namespace de
