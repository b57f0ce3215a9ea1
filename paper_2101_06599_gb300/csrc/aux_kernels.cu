// aux_kernels.cu — initial population, whole-population evaluation, best
// tracking helpers and slot normalisation.
#include <algorithm>

#include "gen_kernel.cuh"
#include "internal.h"

namespace de {

// Test hook: Eq. (9)'s L and Alg. 8's continuation test for caller-given
// words, through the device functions the generation kernels use: the NEC
// lookup on the table in global memory (row-per-CTA and streaming kernels)
// and on the table staged in shared memory (pipelined kernel, batched plans),
// when it fits kDebugTableCap entries, else through global memory as those
// kernels then do.
constexpr int kDebugTableCap = 4096;

__global__ void debug_lengths_kernel(const __grid_constant__ GenParams p, const uint32_t* __restrict__ words, int n,
                                     int* L_global, int* L_shared, uint8_t* exp_cont) {
  __shared__ uint32_t tab[kDebugTableCap];
  const bool staged = p.nT <= kDebugTableCap;
  if (staged)
    for (int k = threadIdx.x; k < p.nT; k += blockDim.x) tab[k] = p.nec_tm1[k];
  __syncthreads();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t w = words[k];
    if (L_global) L_global[k] = nec_length_of<false>(p, w, p.nec_tm1);
    if (L_shared) L_shared[k] = staged ? nec_length_of<true>(p, w, tab) : nec_length_of<false>(p, w, p.nec_tm1);
    if (exp_cont) exp_cont[k] = exp_continues(p, w) ? 1 : 0;
  }
}

// Test hook: the crossover mask of every row for the generation the context
// is at (the one the next step makes), from the draw functions the
// generation kernels use: j_rand from the row's IDX block, L from the NEC
// lookup or Alg. 8's walk, the binomial bits from the row's BIN blocks. One
// warp per row; mask is N x D bytes, 1 where gene j crosses.
__global__ void debug_mask_kernel(const __grid_constant__ GenParams p, int xo, uint8_t* __restrict__ mask) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)(gridDim.x * blockDim.x) >> 5;
  const uint32_t g = (uint32_t)p.st->gen;
  for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < p.N; i += warps) {
    int jrand = 0, L = 0;
    if (lane == 0) {
      RowDraws d;
      draw_donors(p, g, i, d);
      jrand = d.jrand;
      if (xo == kNec) L = nec_length(p, g, i);
      else if (xo == kExp) L = exp_walk_length(p, g, i);
    }
    jrand = __shfl_sync(0xFFFFFFFFu, jrand, 0);
    L = __shfl_sync(0xFFFFFFFFu, L, 0);
    for (int q = lane; q < p.D4; q += 32) {
      const int j0 = 4 * q;
      unsigned m = 0u;
      if (xo == kBin) {
        m = bin_mask(p, philox_block_rk(p.rk, kStreamBin, p.inst, g, (uint32_t)i, (uint32_t)q), q, jrand);
      } else {
        int dd = j0 - jrand;
        if (dd < 0) dd += p.D;
        for (int e = 0; e < 4; ++e) {
          int de = dd + e;
          if (de >= p.D) de -= p.D;
          m |= (de < L) ? (1u << e) : 0u;
        }
      }
      for (int e = 0; e < 4 && j0 + e < p.D; ++e) mask[(size_t)i * p.D + j0 + e] = (uint8_t)((m >> e) & 1u);
    }
  }
}

cudaError_t launch_debug_mask(const GenParams& p, int xo, uint8_t* mask, cudaStream_t s) {
  const int grid = std::max(1, std::min(4096, (p.N + 7) / 8));
  debug_mask_kernel<<<grid, 256, 0, s>>>(p, xo, mask);
  return cudaGetLastError();
}

cudaError_t launch_debug_lengths(const GenParams& p, const uint32_t* words, int n, int* L_global, int* L_shared,
                                 uint8_t* exp_cont, cudaStream_t s) {
  const int grid = std::max(1, std::min(1024, (n + 255) / 256));
  debug_lengths_kernel<<<grid, 256, 0, s>>>(p, words, n, L_global, L_shared, exp_cont);
  return cudaGetLastError();
}

// Alg. 2, first lines: x_ij = clip(lo + (hi - lo) * u_ij), u_ij = (w >> 8) 2^-24,
// with w = word j of the row's INIT stream; each operation rounded once.
__global__ void init_kernel(const __grid_constant__ GenParams p) {
  const size_t total = (size_t)p.N * (size_t)p.D4;
  const float range = __fsub_rn(p.hi, p.lo);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / (size_t)p.D4);
    const int q = (int)(idx - (size_t)i * p.D4);
    const uint4 w = philox_block(p.key, kStreamInit, p.inst, 0u, (uint32_t)i, (uint32_t)q);
    float4 v;
    const int j0 = 4 * q;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float u = (float)(word_of(w, (uint32_t)e) >> 8) * (1.0f / 16777216.0f);
      const float xv = clip_box(__fadd_rn(p.lo, __fmul_rn(range, u)), p.lo, p.hi);
      lane_of(v, e) = (j0 + e < p.D) ? xv : 0.0f;
    }
    reinterpret_cast<float4*>(p.pop0 + (size_t)i * p.pitch)[q] = v;
  }
}

template <int OBJ, int V>
__global__ void __launch_bounds__(kMaxThreads) eval_kernel(const __grid_constant__ GenParams p) {
  __shared__ float red[4][32];
  __shared__ float s_first[(OBJ == kRosenbrock) ? V : 1][32];
  const int i = blockIdx.x;
  const int t = threadIdx.x, T = blockDim.x;
  const long long gen = p.st->gen;
  const int si = p.slots[(size_t)(gen & 1) * p.N + i];
  const float4* xrow = reinterpret_cast<const float4*>((si ? p.pop1 : p.pop0) + (size_t)i * p.pitch);
  float4 x[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int q = t + k * T;
    x[k] = (q < p.D4) ? ld_stream(xrow + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  int cnt = 0;
  const float f = block_row_fitness<OBJ, V>(x, cnt, p, s_first, red);
  if (t == 0) {
    p.fit[i] = f;
    atomicMin(&p.st->best_key, best_key_of(f, i));
  }
}

template <int OBJ>
static cudaError_t launch_eval_obj(int vidx, const GenParams& p, int block, cudaStream_t s) {
  const dim3 grid((unsigned)p.N), blk((unsigned)block);
  switch (vidx) {
    case 0: eval_kernel<OBJ, 1><<<grid, blk, 0, s>>>(p); break;
    case 1: eval_kernel<OBJ, 2><<<grid, blk, 0, s>>>(p); break;
    case 2: eval_kernel<OBJ, 4><<<grid, blk, 0, s>>>(p); break;
    case 3: eval_kernel<OBJ, 8><<<grid, blk, 0, s>>>(p); break;
    case 4: eval_kernel<OBJ, 16><<<grid, blk, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_eval(int obj, int vidx, const GenParams& p, int block, cudaStream_t s) {
  switch (obj) {
    case kSphere: return launch_eval_obj<kSphere>(vidx, p, block, s);
    case kRastrigin: return launch_eval_obj<kRastrigin>(vidx, p, block, s);
    case kAckley: return launch_eval_obj<kAckley>(vidx, p, block, s);
    case kRosenbrock: return launch_eval_obj<kRosenbrock>(vidx, p, block, s);
    case kGriewank: return launch_eval_obj<kGriewank>(vidx, p, block, s);
    case kElliptic: return launch_eval_obj<kElliptic>(vidx, p, block, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void reset_best_kernel(DevState* st) { st->best_key = ~0ULL; }

__global__ void best_from_fit_kernel(const __grid_constant__ GenParams p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x) {
    float f = p.fit[i];
    if (f != f) {
      f = __int_as_float(0x7F800000);
      p.fit[i] = f;
    }
    atomicMin(&p.st->best_key, best_key_of(f, i));
  }
}

__global__ void close_eval_kernel(DevState* st) {
  st->best_f = from_ordered_bits((uint32_t)(st->best_key >> 32));
  st->base_row = (int)(uint32_t)(st->best_key & 0xFFFFFFFFull);
  st->best_gen = st->gen;
  st->done = 0u;
}

// One float4 of the best row per thread (the row is read in one round trip);
// block 0 also writes the header. `out` may be device memory or a mapped,
// page-locked host record.
__global__ void best_gather_kernel(const __grid_constant__ GenParams p, unsigned char* out) {
  griddep_wait();                                  // the generation before it has closed
  griddep_launch_dependents();                     // the next generation's CTAs may take their places
  const unsigned long long bk = p.st->best_key;
  int idx = (int)(uint32_t)(bk & 0xFFFFFFFFull);
  if (idx < 0 || idx >= p.N) idx = 0;   // only before any evaluation
  const long long gen = p.st->gen;
  const int si = p.slots[(size_t)(gen & 1) * p.N + idx];
  const float* row = (si ? p.pop1 : p.pop0) + (size_t)idx * p.pitch;
  float* dst = reinterpret_cast<float*>(out + kStagingHeader);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < p.D4) {
    const float4 v = reinterpret_cast<const float4*>(row)[q];
    const int j = 4 * q;
    if (j + 4 <= p.D) {
      reinterpret_cast<float4*>(dst)[q] = v;
    } else {
      dst[j] = v.x;
      if (j + 1 < p.D) dst[j + 1] = v.y;
      if (j + 2 < p.D) dst[j + 2] = v.z;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<double*>(out) = (double)from_ordered_bits((uint32_t)(bk >> 32));
    *reinterpret_cast<long long*>(out + 8) = p.st->best_gen;
    *reinterpret_cast<int*>(out + 16) = idx;
    *reinterpret_cast<int*>(out + 20) = (int)p.st->error;
  }
}

__global__ void normalize_kernel(const __grid_constant__ GenParams p) {
  const int i = blockIdx.x;
  uint8_t* sl = p.slots + (size_t)(p.st->gen & 1) * p.N;
  if (sl[i] == 0) return;
  const float4* src = reinterpret_cast<const float4*>(p.pop1 + (size_t)i * p.pitch);
  float4* dst = reinterpret_cast<float4*>(p.pop0 + (size_t)i * p.pitch);
  for (int q = threadIdx.x; q < p.D4; q += blockDim.x) dst[q] = src[q];
  __syncthreads();
  if (threadIdx.x == 0) sl[i] = 0;
}

static unsigned grid_for(size_t work, unsigned block) {
  size_t g = (work + block - 1) / block;
  if (g > 152u * 32u) g = 152u * 32u;   // 152 SMs; grid-stride beyond that
  return (unsigned)(g ? g : 1);
}

cudaError_t launch_init(const GenParams& p, cudaStream_t s) {
  init_kernel<<<grid_for((size_t)p.N * p.D4, 256), 256, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_reset_best(const GenParams& p, cudaStream_t s) {
  reset_best_kernel<<<1, 1, 0, s>>>(p.st);
  return cudaGetLastError();
}
cudaError_t launch_best_from_fit(const GenParams& p, cudaStream_t s) {
  best_from_fit_kernel<<<grid_for((size_t)p.N, 256), 256, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_close_eval(const GenParams& p, cudaStream_t s) {
  close_eval_kernel<<<1, 1, 0, s>>>(p.st);
  return cudaGetLastError();
}
cudaError_t launch_best_gather(const GenParams& p, void* staging, cudaStream_t s) {
  return launch_pdl(best_gather_kernel, dim3((unsigned)((p.D4 + 127) / 128)), dim3(128), 0, s, p,
                    static_cast<unsigned char*>(staging));
}
cudaError_t launch_normalize(const GenParams& p, cudaStream_t s) {
  normalize_kernel<<<(unsigned)p.N, 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace de
