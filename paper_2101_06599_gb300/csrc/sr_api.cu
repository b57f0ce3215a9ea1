// sr_api.cu — host side of the shifted-rotated objectives: operands, error
// bound constants, and the launch sequence of one generation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

// Bound constants of the BF16 path.
//
// Both products see the same FP32 a = fl(u - o). The tensor-core product uses
// a = a_hi + a_lo + e_a and R = R_hi + R_lo + E_R (BF16 roundings, unit
// roundoff 2^-8 each, so |a_lo + e_a| <= 2^-8 |a|, |e_a| <= 2^-16 |a|, the
// same for R entrywise) and keeps a_hi R_hi + a_lo R_hi + a_hi R_lo; its
// z differs from R a by rho = -(R_hi e_a + R_lo (a_lo + e_a) + E_R a).
// Accumulation: 3D FP32 additions on the tensor cores (unit 2^-23, which
// allows truncating adds) and D FMAs on the FP32 path (unit 2^-24).
//
// Worst case: |z_bf16,k - z_fp32,k| <= c |a|_2 by Cauchy-Schwarz (rows of R
// have norm 1), c = 3.05 2^-16 + gamma_3D(2^-23) + gamma_D(2^-24).
//
// Probabilistic (Hoeffding's inequality over independent zero-mean rounding
// errors): sum_k g'(z_k) rho_k has standard deviation at most
// sqrt(3) 1.005 2^-16 max|a_j| |g'|_2 (each of the three residual vectors,
// |R_hi|_2 <= 1.005); the accumulation terms at most
// |g'|_2 c_rw |a|_2 sqrt(3 u_tc^2 + u^2) when the partial sums stay within
// c_rw |a|_2 / sqrt(D), c_rw = 4; the g evaluations (<= 12 roundings each)
// and the sums of D values and nct partials on both paths at most
// u |f| (sqrt(2 (D + nct)) + 12) because every g is >= 0. The tensor cores'
// accumulator truncates: 3D / 16 MMA steps (K = 16 each) round each z_k
// toward zero by at most 2^-23 |z_k| (partial sums taken no larger than
// |z_k|), a bias of at most (3D/16) 2^-23 sum_k |g'(z_k)| |z_k|, which is at
// most n (2 n + 20 pi sqrt(D)) for Rastrigin and 2 |f| for the elliptic
// function. The second-order term is bounded by max|g''| / 2 times twice the
// mean of |dz|_2^2.
static SrBound make_bound(int D, int obj, double ell_k, int kind, double sigmas, double amax, int nct) {
  SrBound b{};
  const double u = std::ldexp(1.0, -24), utc = std::ldexp(1.0, -23);
  b.mode = (kind == DE_BOUND_WORST_CASE) ? 1 : 0;
  const double n3 = 3.0 * D;
  const double g3 = n3 * utc / (1.0 - n3 * utc), g1 = D * u / (1.0 - D * u);
  const double split = 3.05 * std::ldexp(1.0, -16);
  b.delta_per_norm = (float)((split + g3 * (1.0 + 3.0 * std::ldexp(1.0, -8)) + g1) * 1.001);
  // reductions of sum g: 64 terms per column tile plus the tiles, on both paths
  b.rel = (float)(2.0 * (64.0 + D / 64.0 + 8.0) * u + 1e-6);
  double sw = 0.0;
  if (obj == DE_OBJ_SR_ELLIPTIC)
    for (int k = 0; k < D; ++k) sw += std::exp2((double)k * ell_k);
  b.sum_w = (float)sw;

  const double pi = 3.14159265358979323846, c_rw = 4.0;
  const double acc2 = 3.0 * utc * utc + u * u;
  const double g2half = (obj == DE_OBJ_SR_ELLIPTIC) ? std::exp2((double)(D - 1) * ell_k)   // w_max
                                                     : 1.0 + 20.0 * pi * pi;               // (2 + 40 pi^2) / 2
  b.lambda = (float)(sigmas > 0.0 ? sigmas : 8.0);
  b.rep_c = (float)(std::sqrt(3.0) * 1.005 * std::ldexp(1.0, -16) * amax * 1.001);
  b.acc_c = (float)(c_rw * std::sqrt(acc2) * 1.001);
  b.eval_c = (float)(u * (std::sqrt(2.0 * (D + nct)) + 12.0) * 1.001);
  b.quad_a = (float)(g2half * 2.0 * D * 3.0 * std::ldexp(1.0, -32) * amax * amax);
  b.quad_b = (float)(g2half * 2.0 * D * acc2 * c_rw * c_rw);
  b.hconst = (float)(20.0 * pi * std::sqrt((double)D));
  b.bias_c = (float)((3.0 * D / 16.0) * utc * 1.001);
  b.wmax = (float)((obj == DE_OBJ_SR_ELLIPTIC) ? std::exp2((double)(D - 1) * ell_k) * 1.0001 : 0.0);
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
  sp.inc_part = (double*)ctx_alloc(c, (size_t)D * sizeof(double));
  sp.inc_count = (unsigned*)ctx_alloc(c, sizeof(unsigned));
  if (!shift || !rot || !sp.part_g || !sp.part_w || !sp.norm2 || !sp.fit_err || !sp.amb || !sp.amb_count ||
      !sp.part2_g || !sp.part2_w || !sp.inc_part || !sp.inc_count)
    return DE_ENOMEM;
  sp.shift = shift;
  sp.rot = rot;
  cudaError_t e = cudaMemcpyAsync(shift, prm->shift, (size_t)D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rot, prm->rotation, (size_t)D * D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.fit_err, 0, (size_t)N * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.amb_count, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.inc_count, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) {
    float* rot_t = (float*)ctx_alloc(c, (size_t)D * D * sizeof(float));
    if (!rot_t) return DE_ENOMEM;
    sp.rot_t = rot_t;
    e = launch_sr_transpose(rot, rot_t, D, c->stream);
  }
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
  double amax = 0.0;                     // max |u_j - o_j| over the box, rounded up
  for (int j = 0; j < D; ++j)
    amax = std::max(amax, std::max(std::fabs((double)c->b.lo - prm->shift[j]), std::fabs((double)c->b.hi - prm->shift[j])));
  amax *= 1.0 + std::ldexp(1.0, -22);
  c->sbound = make_bound(D, c->obj, (double)c->p.ell_k, (int)prm->bound, prm->margin_sigmas, amax, sp.nct);
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
  if (e == cudaSuccess) e = launch_sr_finish(sp, c->incumbent_every, true, c->stream);
  return e;
}

int sr_evaluate(de_ctx* c) {
  SrParams sp = c->sp;
  sp.g = c->p;
  cudaError_t e = launch_reset_best(c->p, c->stream);
  if (e == cudaSuccess) e = launch_sr_gemm_fp32(sp, 1, c->N, c->stream);
  if (e == cudaSuccess) e = launch_sr_store_eval(sp, c->stream);
  if (e == cudaSuccess) e = launch_close_eval(c->p, c->stream);
  if (e == cudaSuccess) e = launch_sr_finish(sp, 1, false, c->stream);
  return cuda_status(e);
}

}  // namespace de_host
