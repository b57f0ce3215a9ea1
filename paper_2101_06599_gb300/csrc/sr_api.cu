// sr_api.cu — host side of the shifted-rotated objectives: operands, error
// bound constants, and the launch sequence of one generation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

// Bound constants for the BF16 path (see the design doc-free derivation here):
// operands split as a = a_hi + a_lo + r_a with |r_a| <= 2^-16 |a| (two BF16
// roundings, unit roundoff 2^-8 each), likewise R; the product keeps a_hi R_hi
// + a_lo R_hi + a_hi R_lo, omitting terms <= 3.05 * 2^-16 |a_j| |R_kj|; the
// 3D-term FP32 accumulation on the tensor cores is bounded by gamma_3D with a
// unit of 2^-23 (truncating adds allowed), the FP32 path's own D-term
// accumulation by gamma_D with 2^-24. Summed over j and with Cauchy-Schwarz
// (rows of R have norm 1): |z_bf16,k - z_fp32,k| <= c |u - o|_2.
static SrBound make_bound(int D, int obj, double ell_k) {
  SrBound b{};
  const double n3 = 3.0 * D, u3 = std::ldexp(1.0, -23), u1 = std::ldexp(1.0, -24);
  const double g3 = n3 * u3 / (1.0 - n3 * u3), g1 = D * u1 / (1.0 - D * u1);
  const double split = 3.05 * std::ldexp(1.0, -16);
  b.delta_per_norm = (float)((split + g3 * (1.0 + 3.0 * std::ldexp(1.0, -8)) + g1) * 1.001);
  // reductions of sum g: 64 terms per column tile plus the tiles, on both paths
  b.rel = (float)(2.0 * (64.0 + D / 64.0 + 8.0) * u1 + 1e-6);
  double sw = 0.0;
  if (obj == DE_OBJ_SR_ELLIPTIC)
    for (int k = 0; k < D; ++k) sw += std::exp2((double)k * ell_k);
  b.sum_w = (float)sw;
  return b;
}

int sr_setup(de_ctx* c, const de_objparams* prm) {
  const int N = c->N, D = c->D;
  SrParams& sp = c->sp;
  std::memset(&sp, 0, sizeof(sp));
  c->rotated = true;
  sp.obj = c->obj;
  sp.prec = (prm->prec == DE_PREC_BF16) ? 2 : 0;
  sp.nct2 = (D + kSrTile - 1) / kSrTile;
  sp.nct = sp.nct2;
  c->incumbent_every = prm->incumbent_every > 0 ? prm->incumbent_every : 50;
  float* shift = (float*)ctx_alloc(c, (size_t)D * sizeof(float));
  float* rot = (float*)ctx_alloc(c, (size_t)D * D * sizeof(float));
  sp.part_g = (float*)ctx_alloc(c, (size_t)N * sp.nct * sizeof(float));
  sp.part_w = (float*)ctx_alloc(c, (size_t)N * sp.nct * sizeof(float));
  sp.norm2 = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  sp.fit_err = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  sp.amb = (int*)ctx_alloc(c, 2 * (size_t)N * sizeof(int));
  sp.amb_count = (unsigned*)ctx_alloc(c, sizeof(unsigned));
  sp.part2_g = (float*)ctx_alloc(c, 2 * (size_t)N * sp.nct2 * sizeof(float));
  sp.part2_w = (float*)ctx_alloc(c, 2 * (size_t)N * sp.nct2 * sizeof(float));
  if (!shift || !rot || !sp.part_g || !sp.part_w || !sp.norm2 || !sp.fit_err || !sp.amb || !sp.amb_count ||
      !sp.part2_g || !sp.part2_w)
    return DE_ENOMEM;
  sp.shift = shift;
  sp.rot = rot;
  cudaError_t e = cudaMemcpyAsync(shift, prm->shift, (size_t)D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rot, prm->rotation, (size_t)D * D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.fit_err, 0, (size_t)N * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.amb_count, 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return DE_ECUDA;
  if (sp.prec == 2) {
    uint16_t* hi = (uint16_t*)ctx_alloc(c, (size_t)D * D * sizeof(uint16_t));
    uint16_t* lo = (uint16_t*)ctx_alloc(c, (size_t)D * D * sizeof(uint16_t));
    sp.a_hi = (uint16_t*)ctx_alloc(c, (size_t)N * D * sizeof(uint16_t));
    sp.a_lo = (uint16_t*)ctx_alloc(c, (size_t)N * D * sizeof(uint16_t));
    if (!hi || !lo || !sp.a_hi || !sp.a_lo) return DE_ENOMEM;
    sp.rot_hi = hi;
    sp.rot_lo = lo;
    if (launch_sr_split_rotation(rot, hi, lo, (size_t)D * D, c->stream) != cudaSuccess) return DE_ECUDA;
    if (prepare_sr_tc() != cudaSuccess) return DE_ECUDA;
    sp.nct = D / 256;                    // one partial per 256-column tile of the tensor-core product
  }
  c->sbound = make_bound(D, c->obj, (double)c->p.ell_k);
  return sync_stream(c);                 // host shift / rotation consumed
}

cudaError_t sr_launch_generation(de_ctx* c, const GenParams& p) {
  SrParams sp = c->sp;
  sp.g = p;
  cudaError_t e = launch_sr_trial(c->xo, c->vidx, sp, c->block, c->stream);
  if (e == cudaSuccess) {
    if (sp.prec == 0) e = launch_sr_gemm_fp32(sp, 0, c->N, c->stream);
    else e = launch_sr_gemm_tc(sp, c->stream);
  }
  if (e == cudaSuccess) e = launch_sr_select(sp, c->sbound, c->stream);
  if (e == cudaSuccess && sp.prec != 0) {
    e = launch_sr_gemm_fp32(sp, 2, 2 * c->N, c->stream);
    if (e == cudaSuccess) e = launch_sr_resolve(sp, c->stream);
  }
  if (e == cudaSuccess) e = launch_sr_close(sp, c->stream);
  if (e == cudaSuccess) e = launch_sr_incumbent(sp, c->incumbent_every, c->stream);
  return e;
}

int sr_evaluate(de_ctx* c) {
  SrParams sp = c->sp;
  sp.g = c->p;
  cudaError_t e = launch_reset_best(c->p, c->stream);
  if (e == cudaSuccess) e = launch_sr_gemm_fp32(sp, 1, c->N, c->stream);
  if (e == cudaSuccess) e = launch_sr_store_eval(sp, c->stream);
  if (e == cudaSuccess) e = launch_close_eval(c->p, c->stream);
  if (e == cudaSuccess) e = launch_sr_incumbent(sp, 1, c->stream);
  return cuda_status(e);
}

}  // namespace de_host
