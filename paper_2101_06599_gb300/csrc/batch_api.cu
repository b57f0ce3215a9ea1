// batch_api.cu — the batched part of the C ABI: many independent DE
// instances advanced together, one generation of all of them per step
// (batch_kernel.cu, batch_stage.cu), and the autotuner of their row kernels.
//
// Device memory: one arena per context holding, per instance, two slot
// buffers (N x pitch floats), fitness, slot bytes and NEC thresholds, plus
// one DevState per instance (contiguous, so the totals are one copy).
// Row work: instance k with G_k <= 32 lanes per row (or the staged kernel)
// is cut into spans of up to 32 rows (one list per row kernel, taken by
// warps from a queue); wider rows are cut into CTA tiles of 256 / G_k rows.
// Lists are grouped by the row code's specialisation, the groups ordered by
// total work (largest first) and the instances longest first within a group.
// A second list of 256-row tiles drives the plan kernel; plans (32 bytes per
// row of every instance) live in one buffer indexed by the instance's first
// row.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

// Lanes per row of the register kernels: the fewest that hold the row in at
// most kBatchMaxD4PerLane float4 slots per lane.
static int min_group(int D4) {
  int G = 4;
  while (G < kBatchMaxGroup && (D4 + G - 1) / G > kBatchMaxD4PerLane) G *= 2;
  return G;
}

// Default row kernel: the staged kernel for the segment crossovers (exp, NEC)
// on rows of D <= 2048 (on the 512-instance NEC mix the fastest single
// choice), register tiles with the fewest lanes otherwise; de_batch_autotune
// refines.
static int default_group(int D4, int xo) {
  if (xo != kBin && D4 <= kStageMaxD4) return kBatchStaged;
  return min_group(D4);
}

static bool valid_group(int G, int D4, int xo) {
  if (G == kBatchStaged) return xo != kBin && D4 <= kStageMaxD4;
  if (G == kBatchFlow) return xo != kBin;
  if (G < 4 || G > kBatchMaxGroup || (G & (G - 1)) != 0) return false;
  return (D4 + G - 1) / G <= kBatchMaxD4PerLane;
}

// Lanes per row in the staged kernel by default: the whole warp (fastest on
// the 512-instance mix for every row length).
static int default_lanes(int) { return 32; }

// The device descriptor of instance k (every field set here, nowhere else).
static BatchInst make_inst(const de_ctx* c, int k) {
  BatchInst bi;
  std::memset(&bi, 0, sizeof(bi));
  bi.g = c->bp[k];
  bi.obj = c->bobj[k];
  bi.xo = c->bxo[k];
  bi.group = c->bgroup[k];
  bi.lanes = c->blanes[k];
  bi.row_base = c->brow_base[k];
  return bi;
}

static int upload_insts(de_ctx* c) {
  std::vector<BatchInst> h((size_t)c->n_inst);
  for (int k = 0; k < c->n_inst; ++k) h[k] = make_inst(c, k);
  if (cudaMemcpyAsync(c->d_insts, h.data(), h.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  return sync_stream(c);
}

// The span list of instance k: register kernel per crossover, staged (3) or
// streaming (4).
static int list_of(const de_ctx* c, int k) {
  if (c->bgroup[k] == kBatchStaged) return 3;
  if (c->bgroup[k] == kBatchFlow) return 4;
  return c->bxo[k];
}

static size_t span_cost(const de_ctx* c, int k) {
  return (size_t)std::min(c->bp[k].N, kSpanRows) * (size_t)c->bp[k].D4;
}

static int upload(de_ctx* c, void** dst, const void* src, size_t bytes) {
  if (*dst) ctx_free(c, *dst);
  *dst = nullptr;
  if (bytes == 0) return DE_OK;
  *dst = ctx_alloc(c, bytes);
  if (!*dst) return DE_ENOMEM;
  return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, c->stream) == cudaSuccess ? DE_OK : DE_ECUDA;
}

static int build_tiles(de_ctx* c) {
  std::vector<int> order((size_t)c->n_inst);
  std::iota(order.begin(), order.end(), 0);
  // instances whose rows take at most a warp go to span lists (one per
  // row kernel), wider rows to CTA tiles of 256 / G rows
  // classes (one specialisation of the row code each) by total work, largest
  // first, so that the warps at the head of the queue share one
  // specialisation as long as possible
  auto cls = [&](int k) {
    const int kind = c->bgroup[k] == kBatchStaged ? 1024 + c->blanes[k] : c->bgroup[k];   // flow: 2
    return (c->bobj[k] * 3 + c->bxo[k]) * 2048 + kind;
  };
  std::map<int, double> work;
  for (int k = 0; k < c->n_inst; ++k) work[cls(k)] += (double)c->bp[k].N * c->bp[k].D4;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ca = cls(a), cb = cls(b);
    if (ca != cb) return work[ca] != work[cb] ? work[ca] > work[cb] : ca < cb;
    return span_cost(c, a) > span_cost(c, b);
  });
  std::vector<BatchSpan> sp[kBatchLists];
  std::vector<BatchTile> ct;
  c->bt0.assign((size_t)c->n_inst, 0);
  c->bt1.assign((size_t)c->n_inst, 0);
  for (int k : order) {
    const int N = c->bp[k].N;
    if (c->bgroup[k] <= 32) {
      std::vector<BatchSpan>& v = sp[list_of(c, k)];
      c->bt0[k] = (int)v.size();
      for (int r = 0; r < N; r += kSpanRows) {
        BatchSpan s;
        std::memset(&s, 0, sizeof(s));
        s.plan0 = c->brow_base[k] + r;
        s.inst = k;
        s.row0 = r;
        s.rows = std::min(kSpanRows, N - r);
        v.push_back(s);
      }
      c->bt1[k] = (int)v.size();
    } else {
      const int R = kBatchThreadsHost / c->bgroup[k];
      c->bt0[k] = (int)ct.size();
      for (int r = 0; r < N; r += R) ct.push_back(BatchTile{k, r});
      c->bt1[k] = (int)ct.size();
    }
  }
  int rc = DE_OK;
  for (int x = 0; x < kBatchLists && rc == DE_OK; ++x) {
    rc = upload(c, (void**)&c->d_spans[x], sp[x].data(), sp[x].size() * sizeof(BatchSpan));
    c->nspans[x] = (int)sp[x].size();
  }
  if (rc == DE_OK) rc = upload(c, (void**)&c->d_ctiles, ct.data(), ct.size() * sizeof(BatchTile));
  c->nctiles = (int)ct.size();
  if (rc != DE_OK) return rc;
  drop_graphs(c);
  return upload_insts(c);
}

// The row work of every instance (inst < 0) or of one instance.
static BatchWork batch_work(const de_ctx* c, int inst) {
  BatchWork w;
  std::memset(&w, 0, sizeof(w));
  w.ctr = c->d_span_ctr;
  w.wait_ns = c->wait_ns;
  if (inst < 0) {
    for (int x = 0; x < kBatchLists; ++x) {
      w.spans[x] = c->d_spans[x];
      w.nspans[x] = c->nspans[x];
    }
    w.ctiles = c->d_ctiles;
    w.nctiles = c->nctiles;
  } else if (c->bgroup[inst] <= 32) {
    const int x = list_of(c, inst);
    w.spans[x] = c->d_spans[x] + c->bt0[inst];
    w.nspans[x] = c->bt1[inst] - c->bt0[inst];
  } else {
    w.ctiles = c->d_ctiles + c->bt0[inst];
    w.nctiles = c->bt1[inst] - c->bt0[inst];
  }
  return w;
}

// Evaluate the parents of every instance (inst < 0) or of one instance.
static int batch_evaluate(de_ctx* c, int inst) {
  const BatchWork w = batch_work(c, inst);
  const cudaError_t e = launch_batch_evaluate(c->d_insts, w, c->d_states, inst < 0 ? 0 : inst,
                                              inst < 0 ? c->n_inst : 1, c->batch_grid, c->stream);
  return cuda_status(e);
}

cudaError_t batch_launch_generation(de_ctx* c, bool, int) {
  const BatchWork w = batch_work(c, -1);
  return launch_batch_generation(c->d_insts, w, c->d_ptiles, c->nptiles, c->d_plans, c->d_states, c->n_inst,
                                 c->batch_grid, c->stream);
}

// Plan tiles: 256 consecutive rows of one instance, instances in order.
static int build_plan_tiles(de_ctx* c) {
  std::vector<BatchTile> pt;
  for (int k = 0; k < c->n_inst; ++k)
    for (int r = 0; r < c->bp[k].N; r += kBatchThreadsHost) pt.push_back(BatchTile{k, r});
  c->d_ptiles = (BatchTile*)ctx_alloc(c, pt.size() * sizeof(BatchTile));
  if (!c->d_ptiles) return DE_ENOMEM;
  c->nptiles = (int)pt.size();
  if (cudaMemcpyAsync(c->d_ptiles, pt.data(), pt.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  return sync_stream(c);
}

int batch_set_base(de_ctx* c, int base) {
  for (int k = 0; k < c->n_inst; ++k) c->bp[k].base = base;
  drop_graphs(c);
  return upload_insts(c);
}

int batch_device_error(de_ctx* c) {
  std::vector<DevState> h((size_t)c->n_inst);
  if (cudaMemcpyAsync(h.data(), c->d_states, h.size() * sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  for (int k = 0; k < c->n_inst; ++k)
    if (h[k].error) return note_device_error(c, (int)h[k].error);
  return DE_OK;
}

int batch_stats(de_ctx* c, de_stats_t* out) {
  std::vector<DevState> h((size_t)c->n_inst);
  if (cudaMemcpyAsync(h.data(), c->d_states, h.size() * sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  std::memset(out, 0, sizeof(*out));
  out->best_f = INFINITY;
  out->best_index = -1;
  out->incumbent_gen = -1;
  out->generation = h.empty() ? 0 : h[0].gen;
  for (int k = 0; k < c->n_inst; ++k) {
    if (h[k].error) return note_device_error(c, (int)h[k].error);
    out->accepts += h[k].accepts;
    out->masked_genes += h[k].masked;
    out->reselected += h[k].reselected;
    if ((double)h[k].best_f < out->best_f) {
      out->best_f = (double)h[k].best_f;
      out->best_index = k;                  // the instance holding the best value
      out->best_gen = h[k].best_gen;
    }
  }
  return DE_OK;
}

}  // namespace de_host

extern "C" {

int de_batch_create(de_ctx** out, int32_t n_inst, const de_instance_spec* specs, uint64_t seed,
                    void* cuda_stream) {
  if (!out) return DE_EINVAL;
  *out = nullptr;
  if (n_inst < 1 || n_inst > (1 << 24) || !specs) return DE_EINVAL;
  for (int k = 0; k < n_inst; ++k) {
    const de_instance_spec& s = specs[k];
    if (!valid_problem(s.N, s.D, s.F, s.CR, (int)s.xo, (int)s.obj, s.b)) return DE_EINVAL;
    if ((int)s.obj > DE_OBJ_ELLIPTIC) return DE_EINVAL;
    if (s.D > 4 * kBatchMaxGroup * kBatchMaxD4PerLane) return DE_EINVAL;
  }
  de_ctx* c = new (std::nothrow) de_ctx();
  if (!c) return DE_ENOMEM;
  c->batch = true;
  c->n_inst = n_inst;
  c->seed = seed;
  c->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  c->batch_grid = std::max(1, c->sm_count) * 2;
  if (prepare_batch_stage() != cudaSuccess || prepare_batch_flow() != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return DE_ECUDA;
  }

  // arena layout
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  std::vector<std::vector<uint32_t>> tabs((size_t)n_inst);
  std::vector<size_t> off_pop0(n_inst), off_pop1(n_inst), off_fit(n_inst), off_slots(n_inst), off_tab(n_inst);
  size_t bytes = a256((size_t)n_inst * sizeof(DevState));
  for (int k = 0; k < n_inst; ++k) {
    const de_instance_spec& s = specs[k];
    const int pitch = ((s.D + 7) / 8) * 8;
    c->max_pitch = std::max(c->max_pitch, pitch);
    tabs[k] = nec_thresholds(s.CR, s.D);
    const size_t pop = (size_t)s.N * pitch * sizeof(float);
    off_pop0[k] = bytes; bytes = a256(bytes + pop);
    off_pop1[k] = bytes; bytes = a256(bytes + pop);
    off_fit[k] = bytes; bytes = a256(bytes + (size_t)s.N * sizeof(float));
    off_slots[k] = bytes; bytes = a256(bytes + 2 * (size_t)s.N);
    off_tab[k] = bytes; bytes = a256(bytes + std::max<size_t>(1, tabs[k].size()) * sizeof(uint32_t));
  }
  unsigned char* arena = (unsigned char*)ctx_alloc(c, bytes);
  c->d_insts = (BatchInst*)ctx_alloc(c, (size_t)n_inst * sizeof(BatchInst));
  c->staging = ctx_alloc(c, kStagingHeader + (size_t)c->max_pitch * sizeof(float));
  c->host_pinned_bytes = std::max(kStagingHeader + (size_t)c->max_pitch * sizeof(float), sizeof(DevState));
  if (!arena || !c->d_insts || !c->staging || cudaMallocHost(&c->host_pinned, c->host_pinned_bytes) != cudaSuccess) {
    cudaGetLastError();
    de_destroy(c);
    return DE_ENOMEM;
  }
  c->d_states = reinterpret_cast<DevState*>(arena);

  c->bp.resize((size_t)n_inst);
  c->bobj.resize((size_t)n_inst);
  c->bxo.resize((size_t)n_inst);
  c->bgroup.resize((size_t)n_inst);
  c->blanes.resize((size_t)n_inst);
  c->bcr.resize((size_t)n_inst);
  c->bF.resize((size_t)n_inst);
  c->bb.resize((size_t)n_inst);
  std::vector<DevState> st0((size_t)n_inst);
  std::memset(st0.data(), 0, st0.size() * sizeof(DevState));
  c->brow_base.resize((size_t)n_inst);
  long long rows = 0;
  for (int k = 0; k < n_inst; ++k) {
    c->brow_base[k] = rows;
    rows += specs[k].N;
  }
  c->d_plans = (RowPlan32*)ctx_alloc(c, (size_t)rows * sizeof(RowPlan32));
  c->d_span_ctr = (unsigned*)ctx_alloc(c, kBatchCounters * sizeof(unsigned));
  if (!c->d_plans || !c->d_span_ctr ||
      cudaMemsetAsync(c->d_span_ctr, 0, kBatchCounters * sizeof(unsigned), c->stream) != cudaSuccess) {
    de_destroy(c);
    return DE_ENOMEM;
  }
  for (int k = 0; k < n_inst; ++k) {
    const de_instance_spec& s = specs[k];
    GenParams& p = c->bp[k];
    std::memset(&p, 0, sizeof(p));
    p.pop0 = reinterpret_cast<float*>(arena + off_pop0[k]);
    p.pop1 = reinterpret_cast<float*>(arena + off_pop1[k]);
    p.fit = reinterpret_cast<float*>(arena + off_fit[k]);
    p.slots = arena + off_slots[k];
    p.st = c->d_states + k;
    p.nec_tm1 = reinterpret_cast<const uint32_t*>(arena + off_tab[k]);
    p.nT = (int)tabs[k].size();
    p.N = s.N;
    p.D = s.D;
    p.pitch = ((s.D + 7) / 8) * 8;
    p.D4 = (s.D + 3) / 4;
    p.F = s.F;
    p.lo = s.b.lo;
    p.hi = s.b.hi;
    p.cr_mode = (s.CR <= 0.0) ? kCrZero : (s.CR >= 1.0 ? kCrOne : kCrGeneral);
    p.cr_t = (unsigned long long)std::ceil(s.CR * 4294967296.0);
    p.cr_lt = (uint32_t)std::min<unsigned long long>(p.cr_t, 0xFFFFFFFFull);
    p.cr_all = p.cr_t > 0xFFFFFFFFull ? 1 : 0;
    p.key = Key2{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
    p.rk = philox_round_keys(p.key);
    p.inst = (uint32_t)k;
    p.ackley_b = 0.2f;
    p.ell_k = (s.D > 1) ? (float)(6.0 * std::log2(10.0) / (double)(s.D - 1)) : 0.0f;
    p.nec_k = nec_guess_factor(s.CR);
    c->bobj[k] = (int)s.obj;
    c->bxo[k] = (int)s.xo;
    c->bgroup[k] = default_group(p.D4, (int)s.xo);
    c->blanes[k] = default_lanes(p.D4);
    c->bcr[k] = s.CR;
    c->bF[k] = s.F;
    c->bb[k] = s.b;
    st0[k].best_key = ~0ULL;
    st0[k].best_f = INFINITY;
  }
  cudaError_t e = cudaMemsetAsync(arena, 0, bytes, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_states, st0.data(), st0.size() * sizeof(DevState), cudaMemcpyHostToDevice, c->stream);
  for (int k = 0; k < n_inst && e == cudaSuccess; ++k)
    if (!tabs[k].empty())
      e = cudaMemcpyAsync(arena + off_tab[k], tabs[k].data(), tabs[k].size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, c->stream);
  for (int k = 0; k < n_inst && e == cudaSuccess; ++k) e = launch_init(c->bp[k], c->stream);
  int rc = cuda_status(e);
  if (rc == DE_OK) rc = sync_stream(c);              // host tables and states consumed
  if (rc == DE_OK) rc = build_plan_tiles(c);
  if (rc == DE_OK) rc = build_tiles(c);
  if (rc == DE_OK) rc = batch_evaluate(c, -1);
  if (rc == DE_OK) rc = sync_stream(c);
  if (rc != DE_OK) {
    de_destroy(c);
    return rc;
  }
  *out = c;
  return DE_OK;
}

int de_batch_best(de_ctx* c, int32_t inst, float* x_out, double* f_out, int32_t* idx_out,
                  int64_t* best_gen_out) {
  if (!c || !c->batch) return c ? DE_ESTATE : DE_EINVAL;
  if (inst < 0 || inst >= c->n_inst) return DE_EINVAL;
  const GenParams& p = c->bp[inst];
  cudaError_t e = launch_best_gather(p, c->staging, c->stream);
  const size_t bytes = kStagingHeader + (size_t)p.D * sizeof(float);
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
  if (x_out) std::memcpy(x_out, h + kStagingHeader, (size_t)p.D * sizeof(float));
  return DE_OK;
}

int de_batch_stats(de_ctx* c, int32_t inst, de_stats_t* out) {
  if (!c || !out) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  if (inst < 0 || inst >= c->n_inst) return DE_EINVAL;
  DevState s;
  if (cudaMemcpyAsync(c->host_pinned, c->d_states + inst, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return DE_ECUDA;
  const int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  std::memcpy(&s, c->host_pinned, sizeof(s));
  if (s.error) return note_device_error(c, (int)s.error);
  out->generation = s.gen;
  out->accepts = s.accepts;
  out->masked_genes = s.masked;
  out->reselected = s.reselected;
  out->best_gen = s.best_gen;
  out->best_f = (double)s.best_f;
  out->best_index = (int32_t)(uint32_t)(s.best_key & 0xFFFFFFFFull);
  out->incumbent_f64 = 0.0;
  out->incumbent_gen = -1;
  return DE_OK;
}

int de_batch_get_population(de_ctx* c, int32_t inst, float* pop_out, float* fit_out) {
  if (!c) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  if (inst < 0 || inst >= c->n_inst) return DE_EINVAL;
  const GenParams& p = c->bp[inst];
  cudaError_t e = launch_normalize(p, c->stream);
  if (e == cudaSuccess && pop_out)
    e = copy_rows(pop_out, (size_t)p.D * sizeof(float), p.pop0, (size_t)p.pitch * sizeof(float),
                          (size_t)p.D * sizeof(float), (size_t)p.N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && fit_out)
    e = cudaMemcpyAsync(fit_out, p.fit, (size_t)p.N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  return sync_stream(c);
}

int de_batch_set_population(de_ctx* c, int32_t inst, const float* pop, const float* fit) {
  if (!c || !pop) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  if (inst < 0 || inst >= c->n_inst) return DE_EINVAL;
  const GenParams& p = c->bp[inst];
  cudaError_t e = cudaMemsetAsync(p.slots + (size_t)(c->host_gen & 1) * p.N, 0, (size_t)p.N, c->stream);
  if (e == cudaSuccess)
    e = copy_rows(p.pop0, (size_t)p.pitch * sizeof(float), pop, (size_t)p.D * sizeof(float),
                          (size_t)p.D * sizeof(float), (size_t)p.N, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  int rc;
  if (fit) {
    e = cudaMemcpyAsync(p.fit, fit, (size_t)p.N * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_reset_best(p, c->stream);
    if (e == cudaSuccess) e = launch_best_from_fit(p, c->stream);
    if (e == cudaSuccess) e = launch_close_eval(p, c->stream);
    rc = cuda_status(e);
  } else {
    rc = batch_evaluate(c, inst);
  }
  if (rc != DE_OK) return rc;
  return sync_stream(c);
}

int de_batch_debug_step(de_ctx* c, int32_t inst, float* trial_out, float* ftrial_out, uint8_t* accept_out,
                        int32_t* draws_out) {
  if (!c) return DE_EINVAL;
  if (!c->batch || c->failed) return DE_ESTATE;
  if (inst < 0 || inst >= c->n_inst) return DE_EINVAL;
  const GenParams& p0 = c->bp[inst];
  BatchInst bi = make_inst(c, inst);
  float* dtrial = trial_out ? (float*)ctx_alloc(c, (size_t)p0.N * p0.pitch * sizeof(float)) : nullptr;
  float* dft = ftrial_out ? (float*)ctx_alloc(c, (size_t)p0.N * sizeof(float)) : nullptr;
  uint8_t* dacc = accept_out ? (uint8_t*)ctx_alloc(c, (size_t)p0.N) : nullptr;
  int* ddr = draws_out ? (int*)ctx_alloc(c, (size_t)p0.N * 5 * sizeof(int)) : nullptr;
  int rc = DE_OK;
  if ((trial_out && !dtrial) || (ftrial_out && !dft) || (accept_out && !dacc) || (draws_out && !ddr)) rc = DE_ENOMEM;
  cudaError_t e = cudaSuccess;
  if (rc == DE_OK) {
    bi.g.dbg_trial = dtrial;
    bi.g.dbg_ftrial = dft;
    bi.g.dbg_accept = dacc;
    bi.g.dbg_draws = ddr;
    e = cudaMemcpyAsync(c->d_insts + inst, &bi, sizeof(bi), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = batch_launch_generation(c, true, inst);
    if (e == cudaSuccess) c->host_gen++;
    bi.g = p0;   // restore the descriptor without test outputs
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_insts + inst, &bi, sizeof(bi), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && trial_out)
      e = copy_rows(trial_out, (size_t)p0.D * sizeof(float), dtrial, (size_t)p0.pitch * sizeof(float),
                            (size_t)p0.D * sizeof(float), (size_t)p0.N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && ftrial_out)
      e = cudaMemcpyAsync(ftrial_out, dft, (size_t)p0.N * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && accept_out)
      e = cudaMemcpyAsync(accept_out, dacc, (size_t)p0.N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && draws_out)
      e = cudaMemcpyAsync(draws_out, ddr, (size_t)p0.N * 5 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    rc = (e == cudaSuccess) ? sync_stream(c) : DE_ECUDA;
  }
  cudaStreamSynchronize(c->stream);
  if (dtrial) ctx_free(c, dtrial);
  if (dft) ctx_free(c, dft);
  if (dacc) ctx_free(c, dacc);
  if (ddr) ctx_free(c, ddr);
  return rc;
}

int de_batch_set_groups(de_ctx* c, const int32_t* groups) {
  if (!c || !groups) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  std::vector<int> g((size_t)c->n_inst), l = c->blanes;
  for (int k = 0; k < c->n_inst; ++k) {
    int G = groups[k];
    const int D4 = c->bp[k].D4;
    if (G == 0) G = default_group(D4, c->bxo[k]);
    if (G == kBatchFlow) {
      if (!valid_group(G, D4, c->bxo[k])) return DE_EINVAL;
      g[k] = G;
      continue;
    }
    if (G == kBatchStaged) {
      l[k] = default_lanes(D4);
    } else if (G < 0) {                              // staged, -G lanes per row
      const int lanes = -G;
      if (lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32) return DE_EINVAL;
      G = kBatchStaged;
      l[k] = lanes;
    }
    if (!valid_group(G, D4, c->bxo[k])) return DE_EINVAL;
    g[k] = G;
  }
  if (sync_stream(c) != DE_OK) return DE_ECUDA;
  c->bgroup = g;
  c->blanes = l;
  return build_tiles(c);
}

int de_batch_get_groups(de_ctx* c, int32_t* groups) {
  if (!c || !groups) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  for (int k = 0; k < c->n_inst; ++k) groups[k] = c->bgroup[k] == kBatchStaged ? -c->blanes[k] : c->bgroup[k];
  return DE_OK;
}

int de_batch_autotune(de_ctx* c, int32_t reps, int32_t* groups_out) {
  if (!c) return DE_EINVAL;
  if (!c->batch || c->failed) return DE_ESTATE;
  if (reps < 1 || reps > 1000) return DE_EINVAL;
  int rc = sync_stream(c);
  if (rc != DE_OK) return rc;
  // classes: same crossover and D4 octave, rows of at most 512 slots
  std::map<int, std::vector<int>> classes;
  for (int k = 0; k < c->n_inst; ++k) {
    const int D4 = c->bp[k].D4;
    if (D4 > kStageMaxD4) continue;
    int oct = 0;
    while ((2 << oct) <= D4) ++oct;
    classes[c->bxo[k] * 64 + oct].push_back(k);
  }
  // snapshot of what the trial generations change: fitness and instance states
  size_t fit_floats = 0;
  for (int k = 0; k < c->n_inst; ++k) fit_floats += (size_t)c->bp[k].N;
  unsigned char* snap = (unsigned char*)ctx_alloc(c, (size_t)c->n_inst * sizeof(DevState) + fit_floats * 4);
  if (!snap) return DE_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemcpyAsync(snap, c->d_states, (size_t)c->n_inst * sizeof(DevState), cudaMemcpyDeviceToDevice,
                                  c->stream);
  {
    size_t off = (size_t)c->n_inst * sizeof(DevState);
    for (int k = 0; k < c->n_inst && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync(snap + off, c->bp[k].fit, (size_t)c->bp[k].N * 4, cudaMemcpyDeviceToDevice, c->stream);
      off += (size_t)c->bp[k].N * 4;
    }
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess)                               // plans of the current generation, reused by every trial
    e = launch_batch_plans(c->d_insts, c->d_ptiles, c->nptiles, c->d_plans, c->batch_grid, c->stream);
  rc = cuda_status(e);
  // time of the row kernels of one generation of every instance under the
  // current choice (their results do not depend on it: every trial writes
  // the same values, which the snapshot undoes)
  auto trial = [&](float& ms) -> int {
    int r = build_tiles(c);
    if (r != DE_OK) return r;
    const BatchWork w = batch_work(c, -1);
    cudaError_t t = launch_batch_rows(c->d_insts, w, c->d_plans, c->batch_grid, c->stream);
    if (t == cudaSuccess) t = cudaEventRecord(e0, c->stream);
    for (int i = 0; i < reps && t == cudaSuccess; ++i)
      t = launch_batch_rows(c->d_insts, w, c->d_plans, c->batch_grid, c->stream);
    if (t == cudaSuccess) t = cudaEventRecord(e1, c->stream);
    if (t == cudaSuccess) t = cudaEventSynchronize(e1);
    if (t == cudaSuccess) t = cudaEventElapsedTime(&ms, e0, e1);
    return cuda_status(t);
  };
  // start from the fastest of a few whole-batch choices: as they stand, the
  // fewest register lanes, 32 register lanes, the staged kernel with its
  // default lanes where allowed, the streaming kernel where allowed
  if (rc == DE_OK) {
    std::vector<int> bg = c->bgroup, bl = c->blanes;
    float best_t = 0.0f;
    rc = trial(best_t);
    for (int rule = 0; rule < 4 && rc == DE_OK; ++rule) {
      std::vector<int> g0 = c->bgroup, l0 = c->blanes;
      for (const auto& cl : classes)
        for (int k : cl.second) {
          const int D4 = c->bp[k].D4, xo = c->bxo[k];
          if (rule == 0) c->bgroup[k] = min_group(D4);
          if (rule == 1) c->bgroup[k] = std::max(min_group(D4), 32);
          if (rule == 2 && valid_group(kBatchStaged, D4, xo)) {
            c->bgroup[k] = kBatchStaged;
            c->blanes[k] = default_lanes(D4);
          }
          if (rule == 3 && valid_group(kBatchFlow, D4, xo)) c->bgroup[k] = kBatchFlow;
          if (!valid_group(c->bgroup[k], D4, xo)) c->bgroup[k] = g0[k];
        }
      float ms = 0.0f;
      rc = trial(ms);
      if (rc == DE_OK && ms < best_t) {
        best_t = ms;
        bg = c->bgroup;
        bl = c->blanes;
      }
      c->bgroup = g0;
      c->blanes = l0;
    }
    c->bgroup = bg;
    c->blanes = bl;
  }
  // coordinate descent: one class at a time, the others as they stand (the
  // streaming kernel is tried for the whole batch only: a mix with the staged
  // kernel would cost the one-launch generation that either gives alone)
  for (auto it = classes.begin(); it != classes.end() && rc == DE_OK; ++it) {
    const std::vector<int>& ks = it->second;
    const int xo = c->bxo[ks[0]];
    int d4max = 0;
    for (int k : ks) d4max = std::max(d4max, c->bp[k].D4);
    std::vector<std::pair<int, int>> cand;       // (group, staged lanes)
    for (int G = 4; G <= 32; G *= 2)
      if (valid_group(G, d4max, xo)) cand.push_back({G, 0});
    if (valid_group(kBatchStaged, d4max, xo))
      for (int l = 4; l <= 32; l *= 2) cand.push_back({kBatchStaged, l});
    if (cand.size() < 2) continue;
    std::vector<int> g0(ks.size()), l0(ks.size());
    for (size_t u = 0; u < ks.size(); ++u) {
      g0[u] = c->bgroup[ks[u]];
      l0[u] = c->blanes[ks[u]];
    }
    float best_t = 0.0f;
    rc = trial(best_t);                              // the class as it stands
    int best = -1;
    for (size_t ci = 0; ci < cand.size() && rc == DE_OK; ++ci) {
      for (int k : ks) {
        c->bgroup[k] = cand[ci].first;
        if (cand[ci].second) c->blanes[k] = cand[ci].second;
      }
      float ms = 0.0f;
      rc = trial(ms);
      if (rc == DE_OK && ms < best_t) {
        best_t = ms;
        best = (int)ci;
      }
      for (size_t u = 0; u < ks.size(); ++u) {
        c->bgroup[ks[u]] = g0[u];
        c->blanes[ks[u]] = l0[u];
      }
    }
    if (best >= 0)
      for (int k : ks) {
        c->bgroup[k] = cand[best].first;
        if (cand[best].second) c->blanes[k] = cand[best].second;
      }
  }
  // restore the snapshot, then the lists for the chosen kernels
  {
    cudaError_t r2 = cudaMemcpyAsync(c->d_states, snap, (size_t)c->n_inst * sizeof(DevState),
                                     cudaMemcpyDeviceToDevice, c->stream);
    size_t off = (size_t)c->n_inst * sizeof(DevState);
    for (int k = 0; k < c->n_inst && r2 == cudaSuccess; ++k) {
      r2 = cudaMemcpyAsync(c->bp[k].fit, snap + off, (size_t)c->bp[k].N * 4, cudaMemcpyDeviceToDevice, c->stream);
      off += (size_t)c->bp[k].N * 4;
    }
    if (rc == DE_OK) rc = cuda_status(r2);
  }
  const int rs = sync_stream(c);
  if (rc == DE_OK) rc = rs;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ctx_free(c, snap);
  const int rb = build_tiles(c);
  if (rc == DE_OK) rc = rb;
  if (rc == DE_OK && groups_out) rc = de_batch_get_groups(c, groups_out);
  return rc;
}

int de_batch_size(de_ctx* c, int32_t* n_inst) {
  if (!c || !n_inst) return DE_EINVAL;
  *n_inst = c->batch ? c->n_inst : 0;
  return DE_OK;
}

}  // extern "C"
