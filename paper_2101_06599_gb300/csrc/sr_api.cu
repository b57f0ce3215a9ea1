// sr_api.cu — host side of the shifted-rotated objectives: operands, error
// bound constants, and the launch sequence of one generation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

using namespace de_host;

namespace de_host {

// Bound constants of the split-operand paths (BF16, FP16).
//
// Both products see the same FP32 a = fl(u - o). The tensor-core product uses
// a = a_hi + a_lo + e_a and R = R_hi + R_lo + E_R, each half a rounding to a
// format of unit roundoff u_s (BF16 2^-8; FP16 2^-11, on 2^sa a and 2^sr R),
// so |a_lo + e_a| <= u_s |a|, |e_a| <= u_s^2 |a| + f_a and |E_R| <= u_s^2 |R|
// + f_r entrywise, where f_a = 2^(-25-sa) and f_r = 2^(-25-sr) are the
// absolute error of a remainder that lands in FP16's subnormal range (zero
// for BF16, which has FP32's range). It keeps a_lo R_hi + a_hi R_lo + a_hi R_hi
// (in that order) and its z differs from R a by
// rho = -(R_hi e_a + R_lo (a_lo + e_a) + E_R a).
// Accumulation: FP32 additions on the tensor cores (unit 2^-23, which allows
// truncating adds): D of the leading product and 2D of the corrections,
// whose partial sums are at most 2.01 u_s of the leading product's; D FMAs
// on the FP32 path (unit 2^-24).
//
// Worst case: |z_split,k - z_fp32,k| <= c |a|_2 + 1.005 f_a sqrt(D) by
// Cauchy-Schwarz (rows of R have norm 1), c = 3.05 u_s^2 + f_r sqrt(D) +
// gamma_3D(2^-23) (1 + 3 u_s) + gamma_D(2^-24).
//
// Probabilistic (Hoeffding's inequality over independent zero-mean rounding
// errors): sum_k g'(z_k) rho_k has standard deviation at most
// sqrt(3) (1.005 u_s^2 max|a_j| + f_a + f_r sqrt(D) max|a_j|) |g'|_2 (each of
// the three residual vectors, |R_hi|_2 <= 1.005; max|a_j| the row's own, which
// the trial kernel records); the accumulation terms at
// most |g'|_2 c_rw |a|_2 sqrt(u_tc^2 (1 + 2 (2.01 u_s)^2) + u^2) when the
// partial sums stay within c_rw |a|_2 / sqrt(D), c_rw = 4; the g evaluations
// and the sums of D values and their tile partials on both
// paths: each g carries at most 12 roundings (12 u g, summed: 12 u |f|, every
// g being >= 0), and each FP32 addition of the sums errs by at most u times
// its partial sum. The FP32 path adds 63 values inside each 64-column tile
// (partials within the tile's sum T_c; sum_c T_c^2 <= f_FP32^2 <= 1.21 f^2,
// the two values of a row being far closer than 10 %)
// and nct2 tile sums (partials within f_FP32); the split path adds 256
// values per 256-column tile (partials within that tile's sum T'_c, known to
// the selection) and nct tile sums. So the sums' deviation is at most
// u sqrt(((63 + nct2) 1.21 + nct) f^2 + 256 sum_c T'_c^2). The tensor
// cores' accumulator truncates: under the same model a truncation error is
// uniform between zero and one ulp toward zero, so the leading product's
// D / 16 MMA steps (K = 16 each) shift each z_k toward zero by half an ulp,
// at most 2^-24 |z_k| (partial sums taken no larger than |z_k|), on average,
// a bias of at most (D/16) 2^-24 sum_k |g'(z_k)| |z_k|, which is at most
// n (2 n + 20 pi sqrt(D)) for Rastrigin and 2 |f| for the elliptic function,
// while the errors' fluctuation about that mean is inside the accumulation
// term; the corrections' 2D / 16 steps, with partial sums within
// 2.01 u_s c_rw n / sqrt(D), add at most (2D/16) 2^-24 2.01 u_s c_rw n |g'|_2.
// The second-order term is bounded by max|g''| / 2 times twice the mean of
// |dz|_2^2.
static SrBound make_bound(int D, int obj, double ell_k, int kind, double sigmas, int nct, double us, double fa,
                          double fr) {
  SrBound b{};
  const double u = std::ldexp(1.0, -24), utc = std::ldexp(1.0, -23);
  const double us2 = us * us, sD = std::sqrt((double)D);
  b.mode = (kind == DE_BOUND_WORST_CASE) ? 1 : 0;
  const double n3 = 3.0 * D;
  const double g3 = n3 * utc / (1.0 - n3 * utc), g1 = D * u / (1.0 - D * u);
  const double split = 3.05 * us2 + fr * sD;
  b.delta_per_norm = (float)((split + g3 * (1.0 + 3.0 * us) + g1) * 1.001);
  b.delta_abs = (float)(1.005 * fa * sD * 1.001);
  // reductions of sum g: 64 terms per column tile plus the tiles, on both paths
  b.rel = (float)(2.0 * (64.0 + D / 64.0 + 8.0) * u + 1e-6);
  double sw = 0.0;
  if (obj == DE_OBJ_SR_ELLIPTIC)
    for (int k = 0; k < D; ++k) sw += std::exp2((double)k * ell_k);
  b.sum_w = (float)sw;

  const double pi = 3.14159265358979323846, c_rw = 4.0;
  const double cs = 2.01 * us;                                       // corrections / leading product
  const double acc2 = utc * utc * (1.0 + 2.0 * cs * cs) + u * u;
  const double g2half = (obj == DE_OBJ_SR_ELLIPTIC) ? std::exp2((double)(D - 1) * ell_k)   // w_max
                                                     : 1.0 + 20.0 * pi * pi;               // (2 + 40 pi^2) / 2
  b.lambda = (float)(sigmas > 0.0 ? sigmas : 8.0);
  b.rep_k = (float)((1.005 * us2 + fr * sD) * 1.001);
  b.rep_f = (float)(fa * 1.001);
  b.acc_c = (float)(c_rw * std::sqrt(acc2) * 1.001);
  const int nct2 = (D + 63) / 64;
  b.eval_c = (float)(u * 12.0 * 1.001);
  b.sum_f2 = (float)((63.0 + nct2) * 1.21 + nct);
  b.sum_t2 = 256.0f;
  b.sum_u = (float)(u * 1.001);
  b.quad_a = (float)(g2half * 2.0 * D * 3.0 * 1.001);
  b.quad_b = (float)(g2half * 2.0 * D * acc2 * c_rw * c_rw);
  b.hconst = (float)(20.0 * pi * sD);
  b.bias_c = (float)((D / 16.0) * 0.5 * utc * 1.001);
  b.bias_c2 = (float)((2.0 * D / 16.0) * 0.5 * utc * cs * c_rw * 1.001);
  b.wmax = (float)((obj == DE_OBJ_SR_ELLIPTIC) ? std::exp2((double)(D - 1) * ell_k) * 1.0001 : 0.0);
  return b;
}

// The power of two s with m 2^s in [2^14, 2^15): FP16 halves of values up to m
// stay below 2^15, and the remainders of values above m 2^-11 stay normal.
static int fp16_scale_exp(double m) {
  if (!(m > 0.0)) return 0;
  int s = 14 - (int)std::floor(std::log2(m));
  while (std::ldexp(m, s) >= 32768.0) --s;
  while (std::ldexp(m, s) < 16384.0) ++s;
  return s;
}

int sr_setup(de_ctx* c, const de_objparams* prm) {
  const int N = c->N, D = c->D;
  SrParams& sp = c->sp;
  std::memset(&sp, 0, sizeof(sp));
  c->rotated = true;
  sp.obj = c->obj;
  sp.prec = (prm->prec == DE_PREC_BF16) ? 2 : (prm->prec == DE_PREC_FP16 ? 3 : 0);
  sp.a_scale = 1.0f;
  sp.z_scale = 1.0f;
  sp.nct2 = (D + kSrTile - 1) / kSrTile;
  sp.nct = sp.nct2;
  c->incumbent_every = prm->incumbent_every > 0 ? prm->incumbent_every : 50;
  float* shift = (float*)ctx_alloc(c, (size_t)D * sizeof(float));
  float* rot = (float*)ctx_alloc(c, (size_t)D * D * sizeof(float));
  sp.part_g = (float*)ctx_alloc(c, (size_t)N * sp.nct * sizeof(float));
  sp.part_w = (float*)ctx_alloc(c, (size_t)N * sp.nct * sizeof(float));
  sp.norm2 = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  sp.amax = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  sp.fit_err = (float*)ctx_alloc(c, (size_t)N * sizeof(float));
  sp.amb = (int*)ctx_alloc(c, 2 * (size_t)N * sizeof(int));
  sp.amb_count = (unsigned*)ctx_alloc(c, sizeof(unsigned));
  sp.part2_g = (float*)ctx_alloc(c, 2 * (size_t)N * sp.nct2 * sizeof(float));
  sp.part2_w = (float*)ctx_alloc(c, 2 * (size_t)N * sp.nct2 * sizeof(float));
  sp.inc_part = (double*)ctx_alloc(c, (size_t)D * sizeof(double));
  sp.inc_count = (unsigned*)ctx_alloc(c, sizeof(unsigned));
  sp.finish_due = (int*)ctx_alloc(c, sizeof(int));
  sp.inc_every = c->incumbent_every;
  if (!shift || !rot || !sp.part_g || !sp.part_w || !sp.norm2 || !sp.amax || !sp.fit_err || !sp.amb || !sp.amb_count ||
      !sp.part2_g || !sp.part2_w || !sp.inc_part || !sp.inc_count || !sp.finish_due)
    return DE_ENOMEM;
  sp.shift = shift;
  sp.rot = rot;
  cudaError_t e = cudaMemcpyAsync(shift, prm->shift, (size_t)D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rot, prm->rotation, (size_t)D * D * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.fit_err, 0, (size_t)N * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.amb_count, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.inc_count, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.finish_due, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) {
    float* rot_t = (float*)ctx_alloc(c, (size_t)D * D * sizeof(float));
    if (!rot_t) return DE_ENOMEM;
    sp.rot_t = rot_t;
    e = launch_sr_transpose(rot, rot_t, D, c->stream);
  }
  if (e != cudaSuccess) return DE_ECUDA;
  double amax = 0.0;                     // max |u_j - o_j| over the box, rounded up
  for (int j = 0; j < D; ++j)
    amax = std::max(amax, std::max(std::fabs((double)c->b.lo - prm->shift[j]), std::fabs((double)c->b.hi - prm->shift[j])));
  amax *= 1.0 + std::ldexp(1.0, -22);
  double us = std::ldexp(1.0, -8), fa = 0.0, fr = 0.0;
  int sa = 0, sr = 0;
  if (sp.prec == 3) {
    double rmax = 0.0;
    for (size_t k = 0; k < (size_t)D * D; ++k) rmax = std::max(rmax, std::fabs((double)prm->rotation[k]));
    sa = fp16_scale_exp(amax);
    sr = fp16_scale_exp(rmax);
    if (sa < -126 || sa > 127 || sa + sr < -126 || sa + sr > 126) return DE_EUNSUPPORTED;   // scales must be normal
    us = std::ldexp(1.0, -11);
    fa = std::ldexp(1.0, -25 - sa);
    fr = std::ldexp(1.0, -25 - sr);
    sp.a_scale = std::ldexp(1.0f, sa);
    sp.z_scale = std::ldexp(1.0f, -(sa + sr));
  }
  if (sp.prec >= 2) {
    uint16_t* hi = (uint16_t*)ctx_alloc(c, (size_t)D * D * sizeof(uint16_t));
    uint16_t* lo = (uint16_t*)ctx_alloc(c, (size_t)D * D * sizeof(uint16_t));
    sp.a_hi = (uint16_t*)ctx_alloc(c, (size_t)N * D * sizeof(uint16_t));
    sp.a_lo = (uint16_t*)ctx_alloc(c, (size_t)N * D * sizeof(uint16_t));
    if (!hi || !lo || !sp.a_hi || !sp.a_lo) return DE_ENOMEM;
    sp.rot_hi = hi;
    sp.rot_lo = lo;
    if (launch_sr_split_rotation(rot, hi, lo, (size_t)D * D, sp.prec == 3, std::ldexp(1.0f, sr), c->stream) !=
        cudaSuccess)
      return DE_ECUDA;
    if (prepare_sr_tc() != cudaSuccess || prepare_sr_list(&sp.list_ctas) != cudaSuccess) return DE_ECUDA;
    sp.nct = D / 256;                    // one partial per 256-column tile of the tensor-core product
  }
  c->sbound = make_bound(D, c->obj, (double)c->p.ell_k, (int)prm->bound, prm->margin_sigmas, sp.nct, us, fa, fr);
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
