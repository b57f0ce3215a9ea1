// ctx.h — the opaque de_ctx of the C ABI and host helpers shared by the
// single-population API (api.cu) and the batched API (batch_api.cu).
#pragma once
#include <cstddef>
#include <map>
#include <vector>

#include "../../include/de.h"
#include "gen_pipe.cuh"
#include "internal.h"
#include "sr_common.cuh"

using namespace de;

namespace de_host {
struct Block {
  void* ptr;
  size_t bytes;
};
}  // namespace de_host

struct de_ctx {
  int32_t N = 0, D = 0, pitch = 0, D4 = 0;
  float F = 0.f;
  double CR = 0.0;
  int xo = 0, obj = 0;
  de_bounds b{0.f, 0.f};
  uint64_t seed = 0;
  uint32_t inst = 0;
  double ackley_b = 0.2;
  cudaStream_t stream = nullptr;
  int block = 32, vidx = 0;
  // kernel choice: 0 = automatic, 1 = row per CTA, 2 = pipelined (exp / NEC)
  int kernel_req = 0;
  bool use_pipe = false;
  bool use_stream = false;         // streaming warp-per-row kernel (gen_stream.cuh)
  bool pipe_ok = false;
  PipeParams pp{};
  int pipe_grid = 0, pipe_block = 32 + 256;
  int pipe_stages_req = 0;       // 0 = as many as fit
  int pipe_cps = 0;              // CTAs per SM (1 or 2); 0 = automatic
  int smem_per_sm = 0;
  int pp_cps = 1;                // CTAs per SM in use
  size_t pipe_smem = 0;
  int sm_count = 0, smem_optin = 0;
  GenParams p{};
  std::vector<de_host::Block> blocks;
  std::map<int32_t, cudaGraphExec_t> graphs;
  void* staging = nullptr;       // device: best row gather
  void* host_pinned = nullptr;   // host: staging copy and state reads
  size_t host_pinned_bytes = 0;
  long long host_gen = 0;
  // a device error reported by a synchronising call (DE_ETIMEOUT, ...): from
  // then on calls that would launch generations return DE_ESTATE
  int failed = 0;
  unsigned long long wait_ns = 0;   // batched grid-barrier limit (0: the 1 s default)
  // batched contexts (de_batch_create); the fields above then describe nothing
  bool batch = false;
  int n_inst = 0;
  std::vector<GenParams> bp;          // per instance, device pointers into the arena
  std::vector<int> bobj, bxo, bgroup, bt0, bt1;   // objective, crossover, group, span / tile range
  std::vector<int> blanes;                         // lanes per row in the staged kernel
  std::vector<double> bcr;
  std::vector<float> bF;
  std::vector<de_bounds> bb;
  de::BatchInst* d_insts = nullptr;
  de::BatchSpan* d_spans[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // register kernel per crossover, staged, streaming
  int nspans[5] = {0, 0, 0, 0, 0};
  unsigned* d_span_ctr = nullptr;        // 2 queue counters per span list
  de::BatchTile* d_ctiles = nullptr;     // CTA tiles (G > 32)
  de::BatchTile* d_ptiles = nullptr;  // plan tiles: 256 rows of one instance
  de::RowPlan32* d_plans = nullptr;
  int nptiles = 0;
  std::vector<long long> brow_base;
  de::DevState* d_states = nullptr;
  int nctiles = 0, batch_grid = 0, max_pitch = 0;
  // shifted-rotated objectives (sr_api.cu)
  bool rotated = false;
  de::SrParams sp{};
  de::SrBound sbound{};
  int incumbent_every = 50;
  int tc_ok = 0;                     // tcgen05 product available for this D
};



namespace de_host {
// Rows of `width` bytes between pitched buffers: one linear copy when both
// sides are contiguous, a 2D copy otherwise.
inline cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                             cudaMemcpyKind kind, cudaStream_t s) {
  if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * rows, kind, s);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s);
}
int cuda_status(cudaError_t e);
void* ctx_alloc(de_ctx* c, size_t bytes);
void ctx_free(de_ctx* c, void* p);
void drop_graphs(de_ctx* c);
void choose_launch(int D4, int& block, int& vidx);
int sync_stream(de_ctx* c);
// Record a device error seen by a synchronising call (the context then
// refuses launches) and return it.
int note_device_error(de_ctx* c, int err);
// The first non-zero device error word over a batch's instances (synchronises).
int batch_device_error(de_ctx* c);
// NEC thresholds T_n - 1 = ceil(c_n 2^32) - 1, c_1 = Cr, c_n = fl(c_{n-1} Cr),
// up to n = D - 1 or before the first T_n <= 1.
std::vector<uint32_t> nec_thresholds(double CR, int D);
float nec_guess_factor(double CR);
// Validation shared by de_create and de_batch_create (non-rotated objectives).
bool valid_problem(int32_t N, int32_t D, float F, double CR, int xo, int obj, de_bounds b);
int batch_set_base(de_ctx* c, int base);
// Batched contexts (batch_api.cu).
cudaError_t batch_launch_generation(de_ctx* c, bool with_debug_of_inst, int inst);
int batch_stats(de_ctx* c, de_stats_t* out);
// Shifted-rotated objectives (sr_api.cu).
int sr_setup(de_ctx* c, const de_objparams* prm);
cudaError_t sr_launch_generation(de_ctx* c, const GenParams& p);
int sr_evaluate(de_ctx* c);
}  // namespace de_host
