// noalloc.cu — one DE/rand/1/NEC generation on device buffers the caller
// owns, with every piece of scratch memory in a fixed array compiled into
// the library, so that the call allocates nothing.
//
// Who needs this: callers that cannot call cudaMalloc. Examples are plug-ins
// running inside another framework that owns every device allocation and
// only lends buffers, code that must not implicitly synchronise the device
// (cudaMalloc and cudaFree may), and programs that reserve a fixed memory
// budget at start-up and may not grow it afterwards.
//
// Scratch kept in g_noalloc_scratch (fixed size, held by every GPU that loads
// the library until the process exits):
//   [0, 256)                 generation state (counters, best key, CTA-done counter)
//   [256, 256 + 2*65536)     slot bytes, two halves of N
//   [.., + 4*32768)          NEC thresholds T_n - 1, n = 1 .. D - 1
// Every call overwrites the state and the slot bytes; the thresholds are
// rewritten only when (Cr, D) differ from the last call's on that device
// (a host-side record per device), since building them takes up to D - 1
// dependent FP64 products on one thread. Calls that overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <algorithm>
#include <cmath>

#include "../../include/de.h"
#include "gen_kernel.cuh"
#include "internal.h"

namespace de {

constexpr int kNoallocMaxN = 65536;
constexpr int kNoallocMaxD = 32768;
constexpr size_t kNoallocStateBytes = 256;
constexpr size_t kNoallocSlotBytes = 2 * (size_t)kNoallocMaxN;
constexpr size_t kNoallocTableBytes = 4 * (size_t)kNoallocMaxD;
constexpr size_t kNoallocScratchBytes = kNoallocStateBytes + kNoallocSlotBytes + kNoallocTableBytes;
constexpr int kNoallocMaxDevices = 64;

static_assert(sizeof(DevState) <= kNoallocStateBytes, "state must fit its scratch region");

}  // namespace de

static __device__ __align__(256) unsigned char g_noalloc_scratch[de::kNoallocScratchBytes];

namespace de {

// Device address of g_noalloc_scratch per device ordinal, taken once with the
// device current (a host-side name of the array is not a device address).
static void* g_scratch_addr[kNoallocMaxDevices];
static bool g_scratch_ready[kNoallocMaxDevices];
// (Cr, D) of the thresholds the array holds, per device ordinal.
static double g_table_cr[kNoallocMaxDevices];
static int g_table_d[kNoallocMaxDevices];   // 0: no table built yet

// Clears what must start at zero (state, the input half of the slot bytes)
// and, when build_table is set, writes the NEC thresholds T_n - 1 =
// ceil(c_n 2^32) - 1 with c_1 = Cr, c_n = fl(c_{n-1} Cr) in FP64, exactly as
// de_create computes them, and 0 from the first T_n <= 1 on (no word w >= 1
// passes those). The products are a chain: thread 0 forms them, a chunk at a
// time, into shared memory, and all threads turn each chunk into thresholds.
constexpr int kNoallocChunk = 256;

__global__ void noalloc_setup_kernel(unsigned char* scratch, int N, int D, double CR, int cr_mode,
                                     long long gen, int build_table) {
  __shared__ double cbuf[kNoallocChunk];
  DevState* st = reinterpret_cast<DevState*>(scratch);
  uint8_t* slots = scratch + kNoallocStateBytes;
  uint32_t* tab = reinterpret_cast<uint32_t*>(scratch + kNoallocStateBytes + kNoallocSlotBytes);
  if (threadIdx.x == 0) {
    st->best_key = ~0ULL;
    st->gen = gen;
    st->best_gen = gen;
    st->accepts = 0ULL;
    st->masked = 0ULL;
    st->reselected = 0ULL;
    st->done = 0u;
    st->error = 0u;
    st->best_f = __int_as_float(0x7F800000);
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) slots[(size_t)(gen & 1) * N + i] = 0;
  if (!build_table) return;
  __shared__ int s_ended;                           // every entry from this chunk on is 0
  double cn = CR;                                   // c_(base + 1), thread 0's running product
  if (threadIdx.x == 0) s_ended = (cr_mode != kCrGeneral);
  __syncthreads();
  for (int base = 0; base < D - 1; base += kNoallocChunk) {
    const int len = min(kNoallocChunk, D - 1 - base);
    const bool ended = s_ended != 0;
    if (threadIdx.x == 0 && !ended) {
      for (int k = 0; k < len; ++k) {
        cbuf[k] = cn;
        cn = __dmul_rn(cn, CR);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      uint32_t t = 0u;
      if (!ended) {
        const double Tn = ceil(__dmul_rn(cbuf[k], 4294967296.0));
        t = (Tn > 1.0) ? (uint32_t)(Tn - 1.0) : 0u;   // T_n <= 1: no word w >= 1 passes
      }
      tab[base + k] = t;
    }
    // the products only decrease: once one is at most 2^-32, every later T_n is at most 1
    if (threadIdx.x == 0 && !ended && cbuf[len - 1] <= 0x1p-32) s_ended = 1;
    __syncthreads();
  }
}

// Rows whose trial was rejected keep the parent: copy it to the output.
__global__ void noalloc_keep_parents_kernel(const float* pop_in, float* pop_out, const uint8_t* slot_out,
                                            int D4, int pitch) {
  const int i = blockIdx.x;
  if (slot_out[i] != 0) return;   // accepted: the generation kernel wrote the trial
  const float4* src = reinterpret_cast<const float4*>(pop_in + (size_t)i * pitch);
  float4* dst = reinterpret_cast<float4*>(pop_out + (size_t)i * pitch);
  for (int q = threadIdx.x; q < D4; q += blockDim.x) dst[q] = src[q];
}

// Launch shape of the row-per-CTA kernel: the rule de_create uses by default
// (smallest float4-per-thread count whose thread count fits 256, else 512).
static void noalloc_shape(int D4, int& block, int& vidx) {
  for (int limit : {256, 512}) {
    for (int k = 0; k < 5; ++k) {
      const int V = kVecChoices[k];
      const int T = (((D4 + V - 1) / V) + 31) / 32 * 32;
      if (T <= limit) {
        block = T;
        vidx = k;
        return;
      }
    }
  }
  block = 512;
  vidx = 4;
}

}  // namespace de

using namespace de;

extern "C" int de_nec_step_noalloc(const float* pop_in, const float* fit_in, float* pop_out, float* fit_out,
                                   int32_t N, int32_t D, int32_t pitch, float F, double CR, de_objective obj,
                                   de_bounds b, uint64_t seed, int64_t generation, void* cuda_stream) {
  if (!pop_in || !fit_in || !pop_out || !fit_out) return DE_EINVAL;
  if (N < 4 || N > kNoallocMaxN || D < 1 || D > kNoallocMaxD) return DE_EINVAL;
  if (pitch < D || pitch % 4 != 0) return DE_EINVAL;
  if (((uintptr_t)pop_in | (uintptr_t)pop_out) % 16 != 0) return DE_EINVAL;
  if (pop_in == pop_out || fit_in == fit_out) return DE_EINVAL;
  if (!std::isfinite(F) || !(CR >= 0.0 && CR <= 1.0) || generation < 0) return DE_EINVAL;
  if ((int)obj < DE_OBJ_SPHERE || (int)obj > DE_OBJ_ELLIPTIC) return DE_EINVAL;
  if (!std::isfinite(b.lo) || !std::isfinite(b.hi) || !(b.lo < b.hi)) return DE_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return DE_ECUDA;
  if (!g_scratch_ready[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) {
      cudaGetLastError();
      return DE_ECUDA;
    }
    g_scratch_addr[dev] = addr;
    g_scratch_ready[dev] = true;
  }
  unsigned char* scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  GenParams p{};
  p.pop0 = const_cast<float*>(pop_in);   // every slot byte is 0: rows are only read from here
  p.pop1 = pop_out;                      // accepted trials are written here
  p.fit = fit_out;
  p.slots = scratch + kNoallocStateBytes;
  p.st = reinterpret_cast<DevState*>(scratch);
  p.nec_tm1 = reinterpret_cast<const uint32_t*>(scratch + kNoallocStateBytes + kNoallocSlotBytes);
  p.nT = D - 1;
  p.N = N;
  p.D = D;
  p.pitch = pitch;
  p.D4 = (D + 3) / 4;
  p.F = F;
  p.lo = b.lo;
  p.hi = b.hi;
  p.cr_mode = (CR <= 0.0) ? kCrZero : (CR >= 1.0 ? kCrOne : kCrGeneral);
  p.cr_t = (unsigned long long)std::ceil(CR * 4294967296.0);
  p.cr_lt = (uint32_t)std::min<unsigned long long>(p.cr_t, 0xFFFFFFFFull);
  p.cr_all = p.cr_t > 0xFFFFFFFFull ? 1 : 0;
  p.key = Key2{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
  p.rk = philox_round_keys(p.key);
  p.inst = 0;
  p.ackley_b = 0.2f;
  p.ell_k = (D > 1) ? (float)(6.0 * std::log2(10.0) / (double)(D - 1)) : 0.0f;
  p.nec_k = (CR > 0.0 && CR < 1.0) ? (float)(1.0 / -std::log2(CR)) : 0.0f;

  int block = 32, vidx = 0;
  noalloc_shape(p.D4, block, vidx);
  const bool build_table = !(g_table_d[dev] == D && g_table_cr[dev] == CR);
  noalloc_setup_kernel<<<1, 256, 0, s>>>(scratch, N, D, CR, p.cr_mode, (long long)generation, build_table ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (build_table) {
    // recorded only once the build is queued; a failed launch builds it again next time
    g_table_d[dev] = (e == cudaSuccess) ? D : 0;
    g_table_cr[dev] = CR;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(fit_out, fit_in, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_gen_nec((int)obj, vidx, p, block, s);
  if (e == cudaSuccess) {
    noalloc_keep_parents_kernel<<<(unsigned)N, 128, 0, s>>>(
        pop_in, pop_out, p.slots + (size_t)((generation + 1) & 1) * N, p.D4, pitch);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? DE_OK : DE_ECUDA;
}
