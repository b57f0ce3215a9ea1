// batch_api.cu — the batched part of the C ABI: many independent DE
// instances advanced by one kernel launch per generation (batch_kernel.cu).
//
// Device memory: one arena per context holding, per instance, two slot
// buffers (N x pitch floats), fitness, slot bytes and NEC thresholds, plus
// one DevState per instance (contiguous, so the totals are one copy).
// Tiles: instance k is cut into ceil(N_k / R_k) tiles, R_k = 32 / G_k rows
// (warp tiles, G_k <= 32) or 256 / G_k rows (CTA tiles); each tile list is
// grouped by (objective, crossover) and ordered by tile cost (R_k D_k,
// descending) within a group, a longest-processing-time schedule for the
// grid-stride walk. A second list
// of 256-row tiles drives the plan kernel; plans (32 bytes per row of every
// instance) live in one buffer indexed by the instance's first row.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

static int default_group(int D4) {
  int G = 4;
  while (G < kBatchMaxGroup && (D4 + G - 1) / G > kBatchMaxD4PerLane) G *= 2;
  return G;
}

// The device descriptor of instance k (every field set here, nowhere else).
static BatchInst make_inst(const de_ctx* c, int k) {
  BatchInst bi;
  std::memset(&bi, 0, sizeof(bi));
  bi.g = c->bp[k];
  bi.obj = c->bobj[k];
  bi.xo = c->bxo[k];
  bi.group = c->bgroup[k];
  bi.tiles = c->bt1[k] - c->bt0[k];
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

static int build_tiles(de_ctx* c) {
  std::vector<int> order((size_t)c->n_inst);
  std::iota(order.begin(), order.end(), 0);
  // grouped by (objective, crossover) so that one specialisation of the row
  // code runs at a time; longest tiles first within a group
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ca = c->bobj[a] * 3 + c->bxo[a], cb = c->bobj[b] * 3 + c->bxo[b];
    if (ca != cb) return ca < cb;
    return (double)(kBatchThreadsHost / c->bgroup[a]) * c->bp[a].D >
           (double)(kBatchThreadsHost / c->bgroup[b]) * c->bp[b].D;
  });
  // rows of G <= 32 lanes go to warp tiles of 32 / G rows, wider rows to CTA
  // tiles of 256 / G rows
  std::vector<BatchTile> wt, ct;
  c->bt0.assign((size_t)c->n_inst, 0);
  c->bt1.assign((size_t)c->n_inst, 0);
  for (int k : order) {
    const bool warp = c->bgroup[k] <= 32;
    std::vector<BatchTile>& tiles = warp ? wt : ct;
    const int R = (warp ? 32 : kBatchThreadsHost) / c->bgroup[k];
    const int nt = (c->bp[k].N + R - 1) / R;
    c->bt0[k] = (int)tiles.size();
    for (int t = 0; t < nt; ++t) tiles.push_back(BatchTile{k, t * R});
    c->bt1[k] = (int)tiles.size();
  }
  if (c->d_tiles) ctx_free(c, c->d_tiles);
  if (c->d_ctiles) ctx_free(c, c->d_ctiles);
  c->d_tiles = nullptr;
  c->d_ctiles = nullptr;
  c->ntiles = (int)wt.size();
  c->nctiles = (int)ct.size();
  if (!wt.empty()) {
    c->d_tiles = (BatchTile*)ctx_alloc(c, wt.size() * sizeof(BatchTile));
    if (!c->d_tiles) return DE_ENOMEM;
    if (cudaMemcpyAsync(c->d_tiles, wt.data(), wt.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return DE_ECUDA;
  }
  if (!ct.empty()) {
    c->d_ctiles = (BatchTile*)ctx_alloc(c, ct.size() * sizeof(BatchTile));
    if (!c->d_ctiles) return DE_ENOMEM;
    if (cudaMemcpyAsync(c->d_ctiles, ct.data(), ct.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return DE_ECUDA;
  }
  drop_graphs(c);
  return upload_insts(c);
}

// Evaluate the parents of every instance (inst < 0) or of one instance.
static int batch_evaluate(de_ctx* c, int inst) {
  cudaError_t e;
  if (inst < 0) {
    e = launch_batch_evaluate(c->d_insts, c->d_tiles, c->ntiles, c->d_ctiles, c->nctiles, c->d_states, 0, c->n_inst,
                              c->batch_grid, c->stream);
  } else {
    const int n = c->bt1[inst] - c->bt0[inst];
    if (c->bgroup[inst] <= 32)
      e = launch_batch_evaluate(c->d_insts, c->d_tiles + c->bt0[inst], n, nullptr, 0, c->d_states, inst, 1,
                                c->batch_grid, c->stream);
    else
      e = launch_batch_evaluate(c->d_insts, nullptr, 0, c->d_ctiles + c->bt0[inst], n, c->d_states, inst, 1,
                                c->batch_grid, c->stream);
  }
  return cuda_status(e);
}

cudaError_t batch_launch_generation(de_ctx* c, bool, int) {
  return launch_batch_generation(c->d_insts, c->d_tiles, c->ntiles, c->d_ctiles, c->nctiles, c->d_ptiles,
                                 c->nptiles, c->d_plans, c->d_states, c->n_inst, c->batch_grid, c->stream);
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
    if (h[k].error) return (int)h[k].error;
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
  if (!c->d_plans) {
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
    p.key = Key2{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
    p.inst = (uint32_t)k;
    p.ackley_b = 0.2f;
    p.ell_k = (s.D > 1) ? (float)(6.0 * std::log2(10.0) / (double)(s.D - 1)) : 0.0f;
    c->bobj[k] = (int)s.obj;
    c->bxo[k] = (int)s.xo;
    c->bgroup[k] = default_group(p.D4);
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
  if (derr) return derr;
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
  if (s.error) return (int)s.error;
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
    e = cudaMemcpy2DAsync(pop_out, (size_t)p.D * sizeof(float), p.pop0, (size_t)p.pitch * sizeof(float),
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
    e = cudaMemcpy2DAsync(p.pop0, (size_t)p.pitch * sizeof(float), pop, (size_t)p.D * sizeof(float),
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
  if (!c->batch) return DE_ESTATE;
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
      e = cudaMemcpy2DAsync(trial_out, (size_t)p0.D * sizeof(float), dtrial, (size_t)p0.pitch * sizeof(float),
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
  std::vector<int> g((size_t)c->n_inst);
  for (int k = 0; k < c->n_inst; ++k) {
    int G = groups[k];
    if (G == 0) G = default_group(c->bp[k].D4);
    if (G < 4 || G > kBatchMaxGroup || (G & (G - 1)) != 0) return DE_EINVAL;
    if ((c->bp[k].D4 + G - 1) / G > kBatchMaxD4PerLane) return DE_EINVAL;
    g[k] = G;
  }
  if (sync_stream(c) != DE_OK) return DE_ECUDA;
  c->bgroup = g;
  return build_tiles(c);
}

int de_batch_get_groups(de_ctx* c, int32_t* groups) {
  if (!c || !groups) return DE_EINVAL;
  if (!c->batch) return DE_ESTATE;
  for (int k = 0; k < c->n_inst; ++k) groups[k] = c->bgroup[k];
  return DE_OK;
}

int de_batch_size(de_ctx* c, int32_t* n_inst) {
  if (!c || !n_inst) return DE_EINVAL;
  *n_inst = c->batch ? c->n_inst : 0;
  return DE_OK;
}

}  // extern "C"
