// api.cu — the C ABI of libde.so (declarations and contracts in include/de.h).
//
// Host responsibilities only: argument validation, device buffers, the
// NEC threshold table, launch-shape choice, CUDA-graph capture of de_run,
// checkpoints. Every step of a generation runs in the device kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

namespace {
de_alloc_fn g_alloc = nullptr;
de_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
}  // namespace

int cuda_status(cudaError_t e) { return e == cudaSuccess ? DE_OK : DE_ECUDA; }

void* ctx_alloc(de_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (g_alloc) {
    p = g_alloc(bytes, (void*)c->stream, g_alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->blocks.push_back({p, bytes});
  return p;
}

void ctx_free(de_ctx* c, void* p) {
  for (size_t k = 0; k < c->blocks.size(); ++k) {
    if (c->blocks[k].ptr == p) {
      if (g_free) g_free(p, c->blocks[k].bytes, (void*)c->stream, g_alloc_user);
      else cudaFree(p);
      c->blocks.erase(c->blocks.begin() + (long)k);
      return;
    }
  }
}

void drop_graphs(de_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Launch shape: T threads (multiple of 32, <= 512) x V float4 slots per
// thread with T * V >= D4. Prefer the smallest V whose T fits in 256
// threads, else in 512.
void choose_launch(int D4, int& block, int& vidx) {
  for (int limit : {256, 512}) {
    for (int k = 0; k < 5; ++k) {
      const int V = kVecChoices[k];
      int T = (D4 + V - 1) / V;
      T = ((T + 31) / 32) * 32;
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

bool is_rotated(int obj) { return obj == DE_OBJ_SR_RASTRIGIN || obj == DE_OBJ_SR_ELLIPTIC; }

std::vector<uint32_t> nec_thresholds(double CR, int D) {
  std::vector<uint32_t> tm1;
  if (CR > 0.0 && CR < 1.0) {
    double cn = CR;
    for (int n = 1; n <= D - 1; ++n) {
      const double Tn = std::ceil(cn * 4294967296.0);
      if (Tn <= 1.0) break;
      tm1.push_back((uint32_t)(Tn - 1.0));
      cn = cn * CR;
    }
  }
  return tm1;
}

// The NEC lookup's first-guess factor 1 / -log2(Cr) (0 outside 0 < Cr < 1,
// where the table is not used).
float nec_guess_factor(double CR) {
  return (CR > 0.0 && CR < 1.0) ? (float)(1.0 / -std::log2(CR)) : 0.0f;
}

bool valid_problem(int32_t N, int32_t D, float F, double CR, int xo, int obj, de_bounds b) {
  if (N < 4 || N > (1 << 29) || D < 1 || D > 32768) return false;
  if ((long long)N * (long long)D >= (1LL << 40)) return false;
  if (!std::isfinite(F) || !(CR >= 0.0 && CR <= 1.0)) return false;
  if (xo < DE_XOVER_BIN || xo > DE_XOVER_NEC) return false;
  if (obj < DE_OBJ_SPHERE || obj > DE_OBJ_SR_ELLIPTIC) return false;
  if (!std::isfinite(b.lo) || !std::isfinite(b.hi) || !(b.lo < b.hi)) return false;
  return true;
}

// Pipelined kernel geometry. Donor span buffers hold the segment lengths
// that occur with probability >= 1e-6 (P(L > n) = Cr^n; longer segments read
// their donor genes from global memory), capped at min(D + 8, 1024) floats.
// Stages: as many as fit in the opt-in shared memory (<= 8), or the
// requested count.
void configure_pipe(de_ctx* c) {
  c->pipe_ok = false;
  if (c->xo == DE_XOVER_BIN || c->rotated || c->sm_count <= 0 || c->smem_optin <= 0) return;
  const int row_floats = 4 * c->D4;
  int need = 16;
  if (c->CR >= 1.0) need = c->D + 8;
  else if (c->CR > 0.0) need = (int)std::min(1.0e6, std::ceil(std::log(1e-6) / std::log(c->CR))) + 16;
  const int segcap = std::max(16, std::min(std::min(((c->D + 3) & ~3) + 8, 1024), (need + 3) & ~3));
  const int stage_floats = ((row_floats + 3 * segcap + 31) / 32) * 32;
  const int tcap = (c->xo == DE_XOVER_NEC && c->p.nT <= kPipeTableCap) ? c->p.nT : 0;
  // Two CTAs per SM share the SM's shared memory (1 KB per CTA is reserved).
  // Automatic: two CTAs (each with its own producer, so the per-row consumer
  // chains of one overlap the other's) when two stages fit in half an SM;
  // else one CTA.
  auto stages_for = [&](int cps) {
    const int budget = (cps == 1) ? c->smem_optin : std::min(c->smem_optin, c->smem_per_sm / cps - 1024);
    for (int s = kPipeMaxStages; s >= 2; --s)
      if (pipe_layout(s, tcap, stage_floats).total <= (unsigned)budget) return s;
    return 0;
  };
  int cps = c->pipe_cps;
  if (cps == 0) cps = (stages_for(2) >= 2) ? 2 : 1;
  int S = stages_for(cps);
  if (S < 2) return;
  c->pp_cps = cps;
  if (c->pipe_stages_req >= 2 && c->pipe_stages_req < S) S = c->pipe_stages_req;
  c->pp.stages = S;
  c->pp.segcap = segcap;
  c->pp.tcap = tcap;
  c->pp.row_floats = row_floats;
  c->pp.stage_floats = stage_floats;
  c->pipe_smem = pipe_layout(S, tcap, stage_floats).total;
  c->pipe_grid = std::min(c->N, c->sm_count * cps);
  if (prepare_gen_pipe(c->xo, c->obj, c->pipe_smem) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c->pipe_ok = true;
}

void resolve_kernel(de_ctx* c) {
  c->use_stream = false;
  if (c->kernel_req == 3) {
    c->use_pipe = false;
    c->use_stream = true;
  } else if (c->kernel_req == 2) {
    c->use_pipe = c->pipe_ok;
  } else if (c->kernel_req == 1) {
    c->use_pipe = false;
  } else {
    c->use_pipe = c->pipe_ok && c->D >= 2048;
    c->use_stream = c->xo == DE_XOVER_BIN && c->D >= 2048;
  }
}

cudaError_t launch_generation(de_ctx* c, const GenParams& p) {
  if (c->batch) return batch_launch_generation(c, false, -1);
  if (c->rotated) return sr_launch_generation(c, p);
  if (c->use_pipe) {
    PipeParams pp = c->pp;
    pp.g = p;
    return launch_gen_pipe(c->xo, c->obj, pp, c->pipe_grid, c->pipe_block, c->pipe_smem, c->stream);
  }
  if (c->use_stream) return launch_gen_stream(c->xo, c->obj, p, c->stream);
  switch (c->xo) {
    case DE_XOVER_BIN: return launch_gen_bin(c->obj, c->vidx, p, c->block, c->stream);
    case DE_XOVER_EXP: return launch_gen_exp(c->obj, c->vidx, p, c->block, c->stream);
    default: return launch_gen_nec(c->obj, c->vidx, p, c->block, c->stream);
  }
}

int evaluate_population(de_ctx* c) {
  if (c->rotated) return sr_evaluate(c);
  cudaError_t e = launch_reset_best(c->p, c->stream);
  if (e == cudaSuccess) e = launch_eval(c->obj, c->vidx, c->p, c->block, c->stream);
  if (e == cudaSuccess) e = launch_close_eval(c->p, c->stream);
  return cuda_status(e);
}

int note_device_error(de_ctx* c, int err) {
  if (err != DE_OK && !c->failed) c->failed = err;
  return err;
}

int sync_stream(de_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  return cuda_status(cudaGetLastError());
}

constexpr uint32_t kSaveMagic = 0x42474544u;   // "DEGB"
constexpr uint32_t kSaveVersion = 1u;

struct SaveHeader {
  uint32_t magic, version;
  int32_t N, D;
  float F, lo, hi, pad0;
  double CR, ackley_b;
  int32_t xo, obj;
  uint64_t seed;
  uint32_t inst, repair;       // repair: 0 in checkpoints written before the field (clip)
  DevState st;
};

}  // namespace

extern "C" {

int de_version(void) { return 100; }

const char* de_strerror(int code) {
  switch (code) {
    case DE_OK: return "ok";
    case DE_EINVAL: return "invalid argument";
    case DE_ENOMEM: return "out of memory";
    case DE_ECUDA: return "CUDA error";
    case DE_ETIMEOUT: return "device-side wait timed out";
    case DE_ESTATE: return "call not valid in this state";
    case DE_EUNSUPPORTED: return "not supported by this build";
    default: return "unknown error";
  }
}

int de_set_allocator(de_alloc_fn alloc, de_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return DE_EINVAL;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return DE_OK;
}

void de_destroy(de_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  while (!c->blocks.empty()) ctx_free(c, c->blocks.back().ptr);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  delete c;
}

int de_create(de_ctx** out, int32_t N, int32_t D, float F, double CR, de_crossover xo,
              de_objective obj, const de_objparams* prm, de_bounds b, uint64_t seed,
              void* cuda_stream) {
  if (!out) return DE_EINVAL;
  *out = nullptr;
  if (!valid_problem(N, D, F, CR, (int)xo, (int)obj, b)) return DE_EINVAL;
  if (is_rotated(obj)) {
    if (!prm || !prm->shift || !prm->rotation) return DE_EINVAL;
    if (prm->bound != DE_BOUND_PROBABILISTIC && prm->bound != DE_BOUND_WORST_CASE) return DE_EINVAL;
    if (!std::isfinite(prm->margin_sigmas) || prm->margin_sigmas < 0.0) return DE_EINVAL;
    if (prm->prec != DE_PREC_FP32 && prm->prec != DE_PREC_BF16 && prm->prec != DE_PREC_FP16) return DE_EUNSUPPORTED;
    if (prm->prec != DE_PREC_FP32 && !sr_tc_supported(D)) return DE_EUNSUPPORTED;
  }
  int repair = DE_REPAIR_CLIP;
  if (prm) {
    if (prm->repair != DE_REPAIR_CLIP && prm->repair != DE_REPAIR_MIDPOINT) return DE_EINVAL;
    repair = (int)prm->repair;
  }
  double ackley_b = 0.2;
  if (prm && prm->ackley_b != 0.0) {
    if (!std::isfinite(prm->ackley_b)) return DE_EINVAL;
    ackley_b = prm->ackley_b;
  }

  de_ctx* c = new (std::nothrow) de_ctx();
  if (!c) return DE_ENOMEM;
  c->N = N;
  c->D = D;
  c->pitch = ((D + 7) / 8) * 8;
  c->D4 = (D + 3) / 4;
  c->F = F;
  c->CR = CR;
  c->xo = (int)xo;
  c->obj = (int)obj;
  c->b = b;
  c->seed = seed;
  c->inst = 0;
  c->ackley_b = ackley_b;
  c->stream = (cudaStream_t)cuda_stream;
  choose_launch(c->D4, c->block, c->vidx);

  // NEC thresholds T_n - 1, T_n = ceil(c_n 2^32), c_1 = Cr, c_n = fl(c_{n-1} Cr);
  // stop before the first T_n <= 1 or at n = D - 1.
  const std::vector<uint32_t> tm1 = nec_thresholds(CR, D);

  const size_t pop_bytes = (size_t)N * (size_t)c->pitch * sizeof(float);
  float* pop0 = (float*)ctx_alloc(c, pop_bytes);
  float* pop1 = (float*)ctx_alloc(c, pop_bytes);
  float* fit = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  uint8_t* slots = (uint8_t*)ctx_alloc(c, 2 * (size_t)N);
  DevState* st = (DevState*)ctx_alloc(c, sizeof(DevState));
  uint32_t* nec = (uint32_t*)ctx_alloc(c, std::max<size_t>(1, tm1.size()) * sizeof(uint32_t));
  c->staging = ctx_alloc(c, kStagingHeader + (size_t)c->pitch * sizeof(float));
  c->host_pinned_bytes = std::max(kStagingHeader + (size_t)c->pitch * sizeof(float), sizeof(DevState));
  if (!pop0 || !pop1 || !fit || !slots || !st || !nec || !c->staging ||
      cudaMallocHost(&c->host_pinned, c->host_pinned_bytes) != cudaSuccess) {
    cudaGetLastError();
    de_destroy(c);
    return DE_ENOMEM;
  }

  GenParams& p = c->p;
  p.pop0 = pop0;
  p.pop1 = pop1;
  p.fit = fit;
  p.slots = slots;
  p.st = st;
  p.nec_tm1 = nec;
  p.nT = (int)tm1.size();
  p.N = N;
  p.D = D;
  p.pitch = c->pitch;
  p.D4 = c->D4;
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
  p.ackley_b = (float)ackley_b;
  p.ell_k = (D > 1) ? (float)(6.0 * std::log2(10.0) / (double)(D - 1)) : 0.0f;
  p.nec_k = nec_guess_factor(CR);
  p.repair = repair;

  c->rotated = is_rotated(obj);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  }
  cudaGetLastError();
  configure_pipe(c);
  resolve_kernel(c);
  if (!c->rotated && prepare_gen_stream(c->xo, c->obj) != cudaSuccess) {
    cudaGetLastError();
    de_destroy(c);
    return DE_ECUDA;
  }

  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.best_key = ~0ULL;
  s0.best_f = INFINITY;
  s0.incumbent_gen = -1;
  int src = DE_OK;
  if (is_rotated(obj)) src = sr_setup(c, prm);
  if (src != DE_OK) {
    de_destroy(c);
    return src;
  }
  cudaError_t e = cudaMemsetAsync(pop0, 0, pop_bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pop1, 0, pop_bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(slots, 0, 2 * (size_t)N, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && !tm1.empty())
    e = cudaMemcpyAsync(nec, tm1.data(), tm1.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_init(p, c->stream);
  int rc = cuda_status(e);
  if (rc == DE_OK) rc = evaluate_population(c);
  // the threshold table lives in pageable memory: make sure it was consumed
  if (rc == DE_OK) rc = sync_stream(c);
  if (rc != DE_OK) {
    de_destroy(c);
    return rc;
  }
  *out = c;
  return DE_OK;
}

int de_step(de_ctx* c) {
  if (!c) return DE_EINVAL;
  if (c->failed) return DE_ESTATE;
  const int rc = cuda_status(launch_generation(c, c->p));
  if (rc == DE_OK) c->host_gen++;
  return rc;
}

// The cached graph of `generations` generations, captured and instantiated on
// first use. Capture records launches without running them, so the context's
// device state is unchanged; nullptr on a CUDA error.
static cudaGraphExec_t run_graph(de_ctx* c, int32_t generations) {
  auto it = c->graphs.find(generations);
  if (it != c->graphs.end()) return it->second;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return nullptr;
  cudaError_t le = cudaSuccess;
  for (int32_t k = 0; k < generations && le == cudaSuccess; ++k) le = launch_generation(c, c->p);
  e = cudaStreamEndCapture(c->stream, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return nullptr;
  c->graphs.emplace(generations, exec);
  return exec;
}

int de_prepare_run(de_ctx* c, int32_t generations) {
  if (!c || generations < 0) return DE_EINVAL;
  if (c->failed) return DE_ESTATE;
  if (generations <= 1 || c->stream == nullptr) return DE_OK;
  return run_graph(c, generations) ? DE_OK : DE_ECUDA;
}

int de_run(de_ctx* c, int32_t generations) {
  if (!c || generations < 0) return DE_EINVAL;
  if (c->failed) return DE_ESTATE;
  if (generations == 0) return DE_OK;
  if (generations == 1 || c->stream == nullptr) {
    for (int32_t k = 0; k < generations; ++k) {
      const int rc = de_step(c);
      if (rc != DE_OK) return rc;
    }
    return DE_OK;
  }
  const cudaGraphExec_t exec = run_graph(c, generations);
  if (!exec) return DE_ECUDA;
  if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) return DE_ECUDA;
  c->host_gen += generations;
  return DE_OK;
}

int de_synchronize(de_ctx* c) {
  if (!c) return DE_EINVAL;
  if (c->batch) return batch_device_error(c);
  if (cudaMemcpyAsync(c->host_pinned, &c->p.st->error, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  unsigned err;
  std::memcpy(&err, c->host_pinned, sizeof(err));
  return note_device_error(c, (int)err);
}

int de_best(de_ctx* c, float* x_out, double* f_out, int32_t* idx_out, int64_t* best_gen_out) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  cudaError_t e = launch_best_gather(c->p, c->staging, c->stream);
  const size_t bytes = kStagingHeader + (size_t)c->D * sizeof(float);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->host_pinned, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  const unsigned char* h = static_cast<const unsigned char*>(c->host_pinned);
  int derr = 0;
  std::memcpy(&derr, h + 20, sizeof(int));
  if (derr) return note_device_error(c, derr);
  if (f_out) std::memcpy(f_out, h, sizeof(double));
  if (best_gen_out) std::memcpy(best_gen_out, h + 8, sizeof(int64_t));
  if (idx_out) std::memcpy(idx_out, h + 16, sizeof(int32_t));
  if (x_out) std::memcpy(x_out, h + kStagingHeader, (size_t)c->D * sizeof(float));
  return DE_OK;
}

int de_best_async(de_ctx* c, void* record_out) {
  if (!c || !record_out) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  // a page-locked record the device can address is written by the gather
  // itself; anything else goes through the staging buffer and a copy
  cudaPointerAttributes a;
  void* dev = nullptr;
  if (((uintptr_t)record_out & 15u) == 0 && cudaPointerGetAttributes(&a, record_out) == cudaSuccess &&
      a.type == cudaMemoryTypeHost && a.devicePointer != nullptr)
    dev = a.devicePointer;
  cudaGetLastError();
  if (dev) return cuda_status(launch_best_gather(c->p, dev, c->stream));
  cudaError_t e = launch_best_gather(c->p, c->staging, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(record_out, c->staging, kStagingHeader + (size_t)c->D * sizeof(float), cudaMemcpyDeviceToHost,
                        c->stream);
  return e == cudaSuccess ? DE_OK : DE_ECUDA;
}

int de_stats(de_ctx* c, de_stats_t* out) {
  if (!c || !out) return DE_EINVAL;
  if (c->batch) return batch_stats(c, out);
  if (cudaMemcpyAsync(c->host_pinned, c->p.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  DevState s;
  std::memcpy(&s, c->host_pinned, sizeof(s));
  if (s.error) return note_device_error(c, (int)s.error);
  out->generation = s.gen;
  out->accepts = s.accepts;
  out->masked_genes = s.masked;
  out->reselected = s.reselected;
  out->best_gen = s.best_gen;
  out->best_f = (double)s.best_f;
  out->best_index = (int32_t)(uint32_t)(s.best_key & 0xFFFFFFFFull);
  out->incumbent_f64 = c->rotated ? s.incumbent_f64 : 0.0;
  out->incumbent_gen = c->rotated ? s.incumbent_gen : -1;
  return DE_OK;
}

int de_get_population(de_ctx* c, float* pop_out, float* fit_out) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  cudaError_t e = launch_normalize(c->p, c->stream);
  if (e == cudaSuccess && pop_out)
    e = copy_rows(pop_out, (size_t)c->D * sizeof(float), c->p.pop0, (size_t)c->pitch * sizeof(float),
                          (size_t)c->D * sizeof(float), (size_t)c->N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && fit_out)
    e = cudaMemcpyAsync(fit_out, c->p.fit, (size_t)c->N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  return sync_stream(c);
}

int de_set_population(de_ctx* c, const float* pop, const float* fit) {
  if (!c || !pop) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  // the current generation's slot half is cleared: buffer 0 holds every row
  cudaError_t e = cudaMemsetAsync(c->p.slots + (size_t)(c->host_gen & 1) * c->N, 0, (size_t)c->N, c->stream);
  if (e == cudaSuccess)
    e = copy_rows(c->p.pop0, (size_t)c->pitch * sizeof(float), pop, (size_t)c->D * sizeof(float),
                          (size_t)c->D * sizeof(float), (size_t)c->N, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  int rc;
  if (fit) {
    e = cudaMemcpyAsync(c->p.fit, fit, (size_t)c->N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->rotated)
      e = cudaMemsetAsync(c->sp.fit_err, 0, (size_t)c->N * sizeof(float), c->stream);
    if (e == cudaSuccess) e = launch_reset_best(c->p, c->stream);
    if (e == cudaSuccess) e = launch_best_from_fit(c->p, c->stream);
    if (e == cudaSuccess) e = launch_close_eval(c->p, c->stream);
    rc = cuda_status(e);
  } else {
    rc = evaluate_population(c);
  }
  if (rc != DE_OK) return rc;
  return sync_stream(c);
}

// Checkpoint layout: header, population (N x D), fitness (N); a shifted-rotated
// context with a split-operand product adds the error bounds of the stored
// fitness values (N), without which a resumed run would take split values as
// exact.
static size_t save_bytes(const de_ctx* c, bool with_err) {
  return sizeof(SaveHeader) + (size_t)c->N * c->D * sizeof(float) + (size_t)c->N * sizeof(float) +
         (with_err ? (size_t)c->N * sizeof(float) : 0);
}

int de_save(de_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return DE_EINVAL;
  if (c->batch) return DE_EUNSUPPORTED;
  const bool with_err = c->rotated && c->sp.prec != 0;
  const size_t need = save_bytes(c, with_err);
  if (!buf) {
    *len = need;
    return DE_OK;
  }
  if (*len < need) return DE_EINVAL;
  unsigned char* o = static_cast<unsigned char*>(buf);
  SaveHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kSaveMagic;
  h.version = kSaveVersion;
  h.N = c->N;
  h.D = c->D;
  h.F = c->F;
  h.lo = c->b.lo;
  h.hi = c->b.hi;
  h.CR = c->CR;
  h.ackley_b = c->ackley_b;
  h.xo = c->xo;
  h.obj = c->obj;
  h.seed = c->seed;
  h.inst = c->inst;
  h.repair = (uint32_t)c->p.repair;
  int rc = de_get_population(c, reinterpret_cast<float*>(o + sizeof(SaveHeader)),
                             reinterpret_cast<float*>(o + sizeof(SaveHeader) + (size_t)c->N * c->D * sizeof(float)));
  if (rc != DE_OK) return rc;
  if (with_err &&
      cudaMemcpyAsync(o + save_bytes(c, false), c->sp.fit_err, (size_t)c->N * sizeof(float), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess)
    return DE_ECUDA;
  if (cudaMemcpyAsync(c->host_pinned, c->p.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  std::memcpy(&h.st, c->host_pinned, sizeof(DevState));
  std::memcpy(o, &h, sizeof(h));
  *len = need;
  return DE_OK;
}

int de_load(de_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return DE_EINVAL;
  if (c->batch) return DE_EUNSUPPORTED;
  if (len < sizeof(SaveHeader)) return DE_EINVAL;
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  // a split-operand context reads the bounds when present (checkpoints written
  // before they were stored have none: their values are then taken as exact)
  const bool with_err = c->rotated && c->sp.prec != 0 && len >= save_bytes(c, true);
  const size_t need = save_bytes(c, with_err);
  if (h.magic != kSaveMagic || h.version != kSaveVersion || len < need) return DE_EINVAL;
  if (h.N != c->N || h.D != c->D || h.F != c->F || h.CR != c->CR || h.xo != c->xo || h.obj != c->obj ||
      h.lo != c->b.lo || h.hi != c->b.hi || h.seed != c->seed || h.inst != c->inst || h.ackley_b != c->ackley_b ||
      h.repair != (uint32_t)c->p.repair)
    return DE_EINVAL;
  if (h.st.gen < 0 || h.st.best_gen < 0 || h.st.best_gen > h.st.gen ||
      (h.st.best_key & 0xFFFFFFFFull) >= (unsigned long long)c->N)
    return DE_EINVAL;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  DevState s = h.st;
  s.done = 0u;
  cudaError_t e = cudaMemcpyAsync(c->p.st, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->p.slots + (size_t)(s.gen & 1) * c->N, 0, (size_t)c->N, c->stream);
  if (e == cudaSuccess)
    e = copy_rows(c->p.pop0, (size_t)c->pitch * sizeof(float), in + sizeof(SaveHeader),
                          (size_t)c->D * sizeof(float), (size_t)c->D * sizeof(float), (size_t)c->N,
                          cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->p.fit, in + sizeof(SaveHeader) + (size_t)c->N * c->D * sizeof(float),
                        (size_t)c->N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && with_err)
    e = cudaMemcpyAsync(c->sp.fit_err, in + save_bytes(c, false), (size_t)c->N * sizeof(float),
                        cudaMemcpyHostToDevice, c->stream);
  else if (e == cudaSuccess && c->rotated)
    e = cudaMemsetAsync(c->sp.fit_err, 0, (size_t)c->N * sizeof(float), c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc == DE_OK) c->host_gen = s.gen;
  return rc;
}

int de_debug_step(de_ctx* c, float* trial_out, float* ftrial_out, uint8_t* accept_out, int32_t* draws_out) {
  if (!c) return DE_EINVAL;
  if (c->failed) return DE_ESTATE;
  if (c->batch) return DE_ESTATE;
  GenParams p = c->p;
  float* dtrial = trial_out ? (float*)ctx_alloc(c, (size_t)c->N * c->pitch * sizeof(float)) : nullptr;
  float* dft = ftrial_out ? (float*)ctx_alloc(c, (size_t)c->N * sizeof(float)) : nullptr;
  uint8_t* dacc = accept_out ? (uint8_t*)ctx_alloc(c, (size_t)c->N) : nullptr;
  int* ddr = draws_out ? (int*)ctx_alloc(c, (size_t)c->N * 5 * sizeof(int)) : nullptr;
  int rc = DE_OK;
  if ((trial_out && !dtrial) || (ftrial_out && !dft) || (accept_out && !dacc) || (draws_out && !ddr)) rc = DE_ENOMEM;
  if (rc == DE_OK) {
    p.dbg_trial = dtrial;
    p.dbg_ftrial = dft;
    p.dbg_accept = dacc;
    p.dbg_draws = ddr;
    rc = cuda_status(launch_generation(c, p));
    if (rc == DE_OK) c->host_gen++;
  }
  cudaError_t e = cudaSuccess;
  if (rc == DE_OK && trial_out)
    e = copy_rows(trial_out, (size_t)c->D * sizeof(float), dtrial, (size_t)c->pitch * sizeof(float),
                          (size_t)c->D * sizeof(float), (size_t)c->N, cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK && e == cudaSuccess && ftrial_out)
    e = cudaMemcpyAsync(ftrial_out, dft, (size_t)c->N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK && e == cudaSuccess && accept_out)
    e = cudaMemcpyAsync(accept_out, dacc, (size_t)c->N, cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK && e == cudaSuccess && draws_out)
    e = cudaMemcpyAsync(draws_out, ddr, (size_t)c->N * 5 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK) rc = (e == cudaSuccess) ? sync_stream(c) : DE_ECUDA;
  else cudaStreamSynchronize(c->stream);
  if (dtrial) ctx_free(c, dtrial);
  if (dft) ctx_free(c, dft);
  if (dacc) ctx_free(c, dacc);
  if (ddr) ctx_free(c, ddr);
  return rc;
}

int de_debug_lengths(de_ctx* c, int32_t inst, const uint32_t* words, int32_t n, int32_t* L_global,
                     int32_t* L_shared, uint8_t* exp_continue) {
  if (!c || n < 0 || (n > 0 && !words)) return DE_EINVAL;
  if (c->batch ? (inst < 0 || inst >= c->n_inst) : inst != 0) return DE_EINVAL;
  if (n == 0) return DE_OK;
  const GenParams& p = c->batch ? c->bp[inst] : c->p;
  uint32_t* dw = (uint32_t*)ctx_alloc(c, (size_t)n * sizeof(uint32_t));
  int* dg = L_global ? (int*)ctx_alloc(c, (size_t)n * sizeof(int)) : nullptr;
  int* ds = L_shared ? (int*)ctx_alloc(c, (size_t)n * sizeof(int)) : nullptr;
  uint8_t* de = exp_continue ? (uint8_t*)ctx_alloc(c, (size_t)n) : nullptr;
  int rc = DE_OK;
  if (!dw || (L_global && !dg) || (L_shared && !ds) || (exp_continue && !de)) rc = DE_ENOMEM;
  cudaError_t e = cudaSuccess;
  if (rc == DE_OK) e = cudaMemcpyAsync(dw, words, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream);
  if (rc == DE_OK && e == cudaSuccess) e = launch_debug_lengths(p, dw, n, dg, ds, de, c->stream);
  if (rc == DE_OK && e == cudaSuccess && L_global)
    e = cudaMemcpyAsync(L_global, dg, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK && e == cudaSuccess && L_shared)
    e = cudaMemcpyAsync(L_shared, ds, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK && e == cudaSuccess && exp_continue)
    e = cudaMemcpyAsync(exp_continue, de, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
  if (rc == DE_OK) rc = (e == cudaSuccess) ? sync_stream(c) : DE_ECUDA;
  else cudaStreamSynchronize(c->stream);
  if (dw) ctx_free(c, dw);
  if (dg) ctx_free(c, dg);
  if (ds) ctx_free(c, ds);
  if (de) ctx_free(c, de);
  return rc;
}

int de_debug_mask(de_ctx* c, int32_t inst, uint8_t* mask_out) {
  if (!c || !mask_out) return DE_EINVAL;
  if (c->batch ? (inst < 0 || inst >= c->n_inst) : inst != 0) return DE_EINVAL;
  const GenParams& p = c->batch ? c->bp[inst] : c->p;
  const int xo = c->batch ? c->bxo[inst] : c->xo;
  const size_t bytes = (size_t)p.N * (size_t)p.D;
  uint8_t* dm = (uint8_t*)ctx_alloc(c, bytes);
  if (!dm) return DE_ENOMEM;
  cudaError_t e = launch_debug_mask(p, xo, dm, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mask_out, dm, bytes, cudaMemcpyDeviceToHost, c->stream);
  const int rc = (e == cudaSuccess) ? sync_stream(c) : DE_ECUDA;
  if (rc != DE_OK) cudaStreamSynchronize(c->stream);
  ctx_free(c, dm);
  return rc;
}

int de_set_wait_limit(de_ctx* c, int64_t ns) {
  if (!c || ns < 0) return DE_EINVAL;
  c->wait_ns = (unsigned long long)ns;
  drop_graphs(c);
  return DE_OK;
}

int de_get_wait_limit(de_ctx* c, int64_t* ns) {
  if (!c || !ns) return DE_EINVAL;
  *ns = c->wait_ns ? (int64_t)c->wait_ns : (int64_t)kWaitLimitNs;
  return DE_OK;
}

int de_set_launch(de_ctx* c, int32_t threads, int32_t vec4) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  int vidx = -1;
  for (int k = 0; k < 5; ++k)
    if (kVecChoices[k] == vec4) vidx = k;
  if (vidx < 0 || threads < 32 || threads > kMaxThreads || threads % 32 != 0) return DE_EINVAL;
  if ((long long)threads * vec4 < c->D4) return DE_EINVAL;
  c->block = threads;
  c->vidx = vidx;
  drop_graphs(c);
  return DE_OK;
}

int de_set_kernel(de_ctx* c, int32_t kind) {
  if (!c || kind < 0 || kind > 3) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  if (kind == 2 && !c->pipe_ok) return DE_EUNSUPPORTED;
  c->kernel_req = kind;
  resolve_kernel(c);
  drop_graphs(c);
  return DE_OK;
}

int de_set_base(de_ctx* c, de_base base) {
  if (!c || (int)base < DE_BASE_DISTINCT || (int)base > DE_BASE_BEST) return DE_EINVAL;
  if (c->batch) return batch_set_base(c, (int)base);
  c->p.base = (int)base;
  drop_graphs(c);
  return DE_OK;
}

int de_get_base(de_ctx* c, de_base* base) {
  if (!c || !base) return DE_EINVAL;
  *base = (de_base)(c->batch ? (c->bp.empty() ? 0 : c->bp[0].base) : c->p.base);
  return DE_OK;
}

int de_get_kernel(de_ctx* c, int32_t* kind) {
  if (!c || !kind) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  *kind = c->use_pipe ? 2 : (c->use_stream ? 3 : 1);
  return DE_OK;
}

int de_set_pipeline(de_ctx* c, int32_t consumer_threads, int32_t stages, int32_t ctas_per_sm) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  if (consumer_threads < 32 || consumer_threads > 32 * kPipeMaxConsumerWarps || consumer_threads % 32 != 0)
    return DE_EINVAL;
  if (stages != 0 && (stages < 2 || stages > kPipeMaxStages)) return DE_EINVAL;
  if (ctas_per_sm < 0 || ctas_per_sm > 2) return DE_EINVAL;
  c->pipe_block = 32 + consumer_threads;
  c->pipe_stages_req = stages;
  c->pipe_cps = ctas_per_sm;
  configure_pipe(c);
  resolve_kernel(c);
  drop_graphs(c);
  return DE_OK;
}

int de_get_pipeline(de_ctx* c, int32_t* consumer_threads, int32_t* stages, int32_t* span_floats,
                    int32_t* ctas_per_sm) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  if (!c->pipe_ok) return DE_EUNSUPPORTED;
  if (ctas_per_sm) *ctas_per_sm = c->pp_cps;
  if (consumer_threads) *consumer_threads = c->pipe_block - 32;
  if (stages) *stages = c->pp.stages;
  if (span_floats) *span_floats = c->pp.segcap;
  return DE_OK;
}

int de_get_launch(de_ctx* c, int32_t* threads, int32_t* vec4) {
  if (!c) return DE_EINVAL;
  if (c->batch) return DE_ESTATE;
  if (threads) *threads = c->block;
  if (vec4) *vec4 = kVecChoices[c->vidx];
  return DE_OK;
}

}  // extern "C"
