// internal.h — host-side launchers of the device kernels (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace de {

// Generation kernels, one translation unit per crossover. vidx indexes
// kVecChoices (float4 slots per thread: 1, 2, 4, 8, 16).
cudaError_t launch_gen_bin(int obj, int vidx, const GenParams& p, int block, cudaStream_t s);
cudaError_t launch_gen_stream(int xo, int obj, const GenParams& p, cudaStream_t s);
cudaError_t prepare_gen_stream(int xo, int obj);
cudaError_t launch_gen_exp(int obj, int vidx, const GenParams& p, int block, cudaStream_t s);
cudaError_t launch_gen_nec(int obj, int vidx, const GenParams& p, int block, cudaStream_t s);

// Uniform initial population into slot buffer 0 (Philox stream INIT).
cudaError_t launch_init(const GenParams& p, cudaStream_t s);
// Fitness of every row (current slots) into fit[], folding each row into
// best_key (reset it first with launch_reset_best).
cudaError_t launch_eval(int obj, int vidx, const GenParams& p, int block, cudaStream_t s);
// best_key <- all ones.
cudaError_t launch_reset_best(const GenParams& p, cudaStream_t s);
// Fold the given fit[] into best_key (after launch_reset_best).
cudaError_t launch_best_from_fit(const GenParams& p, cudaStream_t s);
// best_f <- value of best_key, best_gen <- gen.
cudaError_t launch_close_eval(const GenParams& p, cudaStream_t s);
// staging <- {double f, int64 best_gen, int32 idx, pad, row[D]} of the best row.
cudaError_t launch_best_gather(const GenParams& p, void* staging, cudaStream_t s);
// Move every row held in slot buffer 1 to slot buffer 0 and clear its slot
// bit, so that buffer 0 holds the whole population.
cudaError_t launch_normalize(const GenParams& p, cudaStream_t s);
// Test hook: the N x D crossover mask of the generation the context is at.
cudaError_t launch_debug_mask(const GenParams& p, int xo, uint8_t* mask, cudaStream_t s);
// Test hook: L of Eq. (9) (table in global and in shared memory) and Alg. 8's
// continuation test for n caller-given words (device arrays).
cudaError_t launch_debug_lengths(const GenParams& p, const uint32_t* words, int n, int* L_global, int* L_shared,
                                 uint8_t* exp_cont, cudaStream_t s);

// Pipelined generation kernel (exp / NEC); PipeParams in gen_pipe.cuh.
struct PipeParams;
cudaError_t prepare_gen_pipe(int xo, int obj, size_t smem);
cudaError_t launch_gen_pipe(int xo, int obj, const PipeParams& pp, int grid, int block, size_t smem,
                            cudaStream_t s);

// Batched instances (batch_kernel.cu): one descriptor per instance and a
// tile list; a tile is 256 / group rows of one instance.
struct alignas(16) BatchInst {  // copied into shared memory 16 bytes at a time
  GenParams g;
  int obj, xo;
  int group;                 // lanes per row of the register kernels, or kBatchStaged
  int lanes;                 // lanes per row in the staged kernel (4, 8, 16 or 32)
  long long row_base;        // first plan index of this instance
};
struct BatchTile {
  int inst, row0;
};
// Draws of one row, written by the plan kernel: donors, j_rand, L, the slot
// bytes of the row and its donors (bits 0-7, 8-15, 16-23, 24-31), the
// parent fitness and the parity of the generation being made.
struct RowPlan32 {
  int r1, r2, r3, jrand, L;
  uint32_t slots;
  float fit_i;
  int gpar;
};
// Up to kSpanRows consecutive rows of one instance whose rows take at most
// one warp (G <= 32, or the staged kernel); plan0 = the plan index of row0.
struct alignas(16) BatchSpan {
  long long plan0;
  int inst, row0, rows, pad_[3];
};
constexpr int kSpanRows = 32;
constexpr int kBatchThreadsHost = 256;
constexpr int kBatchMaxGroup = 256;
constexpr int kBatchMaxD4PerLane = 16;
// The row work of one launch: span lists per crossover (bin, exp, NEC) with
// their queue counters (2 per list, zero between launches) and the CTA tiles
// of the instances with G > 32.
struct BatchWork {
  const BatchSpan* spans[5];   // register kernel for bin, exp, NEC; staged kernel, streaming kernel (exp and NEC)
  int nspans[5];
  unsigned* ctr;               // 16 counters (2 per register list; 4 for the staged and the streaming lists)
  unsigned long long wait_ns;  // limit of the one-launch generation's grid barrier (0: 1 s)
  const BatchTile* ctiles;
  int nctiles;
};
// plan kernel + row kernels + close kernel (one generation of every instance)
cudaError_t launch_batch_generation(const BatchInst* insts, const BatchWork& w, const BatchTile* ptiles,
                                    int nptiles, RowPlan32* plans, DevState* states, int n_inst, int grid,
                                    cudaStream_t s);
// the plan kernel alone, and the row kernels alone (plans already made)
cudaError_t launch_batch_plans(const BatchInst* insts, const BatchTile* ptiles, int nptiles, RowPlan32* plans,
                               int grid, cudaStream_t s);
cudaError_t launch_batch_rows(const BatchInst* insts, const BatchWork& w, const RowPlan32* plans, int grid,
                              cudaStream_t s);
// reset best keys, evaluate the parents of the listed rows, close (instances
// first_inst .. first_inst + n_inst - 1)
cudaError_t launch_batch_evaluate(const BatchInst* insts, const BatchWork& w, DevState* states, int first_inst,
                                  int n_inst, int grid, cudaStream_t s);
// the staged row kernel for exp / NEC rows of D <= 2048 (batch_stage.cu)
constexpr int kBatchStaged = 1;          // group value that selects it
constexpr int kStageMaxD4 = 512;
cudaError_t prepare_batch_stage();
cudaError_t launch_batch_stage(const BatchInst*, const BatchSpan*, int, const RowPlan32*, unsigned*, int, int,
                               cudaStream_t);
// one generation of every instance in one cooperative launch when every
// instance is on the staged kernel (plans, rows, close); ctr: 4 counters
bool batch_fused_supported();
cudaError_t launch_batch_fused(const BatchInst* insts, const BatchSpan* spans, int nspans, const BatchTile* ptiles,
                               int nptiles, RowPlan32* plans, DevState* states, int n_inst, unsigned* ctr, int grid,
                               unsigned long long wait_ns, cudaStream_t s);
// the streaming row kernel for exp / NEC rows of any D (batch_flow.cu)
constexpr int kBatchFlow = 2;            // group value that selects it
constexpr int kBatchLists = 5;           // span lists: register bin, exp, NEC; staged; streaming
constexpr int kBatchCounters = 16;
cudaError_t prepare_batch_flow();
cudaError_t launch_batch_flow(const BatchInst*, const BatchSpan*, int, const RowPlan32*, unsigned*, int, int,
                              cudaStream_t);
bool batch_flow_fused_supported();
cudaError_t launch_batch_flow_fused(const BatchInst* insts, const BatchSpan* spans, int nspans,
                                    const BatchTile* ptiles, int nptiles, RowPlan32* plans, DevState* states,
                                    int n_inst, unsigned* ctr, int grid, unsigned long long wait_ns,
                                    cudaStream_t s);
// the span row kernel alone, one per crossover (batch_span_*.cu)
cudaError_t launch_batch_span_bin(const BatchInst*, const BatchSpan*, int, const RowPlan32*, unsigned*, int, int,
                                  cudaStream_t);
cudaError_t launch_batch_span_exp(const BatchInst*, const BatchSpan*, int, const RowPlan32*, unsigned*, int, int,
                                  cudaStream_t);
cudaError_t launch_batch_span_nec(const BatchInst*, const BatchSpan*, int, const RowPlan32*, unsigned*, int, int,
                                  cudaStream_t);

// Shifted-rotated objectives (sr_kernels.cu, sr_tc.cu); SrParams and
// SrBound in sr_common.cuh.
struct SrParams;
struct SrBound;
cudaError_t launch_sr_trial(int xo, int vidx, const SrParams& sp, int block, cudaStream_t s);
cudaError_t launch_sr_gemm_fp32(const SrParams& sp, int mode, int max_rows, cudaStream_t s);
cudaError_t launch_sr_select(const SrParams& sp, const SrBound& b, cudaStream_t s);
cudaError_t launch_sr_resolve(const SrParams& sp, cudaStream_t s);
cudaError_t launch_sr_store_eval(const SrParams& sp, cudaStream_t s);
cudaError_t launch_sr_split_rotation(const float* rot, uint16_t* hi, uint16_t* lo, size_t n, bool fp16, float scale,
                                     cudaStream_t s);
cudaError_t launch_sr_transpose(const float* rot, float* rot_t, int D, cudaStream_t s);
cudaError_t launch_sr_finish(const SrParams& sp, int every, bool close, cudaStream_t s);
// tcgen05 BF16 product (split operands) with the fitness epilogue; requires
// D % 256 == 0. sr_tc_supported tells whether this build and device have it.
cudaError_t launch_sr_gemm_tc(const SrParams& sp, cudaStream_t s);
cudaError_t prepare_sr_tc();
cudaError_t prepare_sr_list(int* ctas);
bool sr_tc_supported(int D);

constexpr size_t kStagingHeader = 32;

}  // namespace de
