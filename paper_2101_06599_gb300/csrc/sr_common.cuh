// sr_common.cuh — shared definitions of the shifted-rotated objective path:
// f(x) = sum_k g(z_k), z = R (x - o), with g the Rastrigin term
// z^2 + 20 sin^2(pi z) (= z^2 - 10 cos 2 pi z + 10) or the elliptic term
// 10^(6k/(D-1)) z_k^2. The product Z = (U - 1 o^T) R^T over a set of rows is
// a GEMM (M = rows, N = K = D); its epilogue reduces g(z) over each column
// tile into per-row partial sums, which a selection kernel adds in a fixed
// order.
#pragma once
#include "common.cuh"
#include "objectives.cuh"

namespace de {

constexpr int kSrTile = 64;          // columns per partial sum of g (both FP32 products)

struct SrParams {
  GenParams g;
  int obj;                 // kSrRastrigin or kSrElliptic
  int prec;                // 0 = FP32, 2 = BF16, 3 = FP16 (split hi/lo operands)
  float a_scale;           // FP16: 2^sa applied to a = u - o before the split (1 otherwise)
  float z_scale;           // FP16: 2^-(sa + sr), undoes both operand scalings on z (1 otherwise)
  int nct;                 // column tiles per row of part_g / part_w (the main product)
  int nct2;                // column tiles per entry of part2_g / part2_w (FP32 product)
  const float* shift;      // o, D floats
  const float* rot;        // R, D x D FP32 row-major (z_k = sum_j R[k][j] a_j)
  const uint16_t* rot_hi;  // hi(R) (BF16, or FP16 of 2^sr R), D x D
  const uint16_t* rot_lo;  // lo(R): the rounded remainder, D x D
  const float* rot_t;      // R transposed (j-major, rot_t[j D + k] = R[k][j]), D x D
  uint16_t* a_hi;          // hi(u - o) (BF16, or FP16 of 2^sa (u - o)), N x D
  uint16_t* a_lo;          // lo(u - o): the rounded remainder, N x D
  float* part_g;           // N x nct: sum of g(z) over the column tile
  float* part_w;           // N x nct: sum of w_k |z_k| (w = 1 Rastrigin, c_k elliptic)
  float* norm2;            // N: |u - o|^2 of the trial (FP32)
  float* amax;             // N: max_j |u_j - o_j| of the trial
  float* fit_err;          // N: bound on |fit - FP32-path value| of the stored parent
  int* amb;                // ambiguous entries: row << 1 | (1 = parent row)
  unsigned* amb_count;     // number of entries in amb
  float* part2_g;          // 2N x nct: partial sums of the re-evaluated entries
  float* part2_w;
  double* inc_part;        // D: FP64 g(z_k) of the incumbent re-evaluation
  unsigned* inc_count;     // CTAs of the incumbent re-evaluation done (last one sums)
  int inc_every;           // FP64 incumbent every inc_every generations
  int* finish_due;         // set by the selection kernel: the incumbent is due at this close
  int list_ctas;           // grid of the ambiguous-entry GEMM: one CTA per SM
};

// Bound constants of the BF16 path (sr_select_kernel). For a row with a =
// u - o, |a|_2 = n and FP32 value f, H bounds |g'(z)|_2: Rastrigin
// min(2 n + 20 pi sqrt(D), (2 + 40 pi^2) n) (|g'(z)| <= 2|z| + 20 pi |sin 2 pi z|
// <= min(2|z| + 20 pi, (2 + 40 pi^2) |z|), |z|_2 = n), elliptic
// 2 sqrt(w_max |f|) (sum w^2 z^2 <= w_max sum w z^2).
struct SrBound {
  int mode;               // 0 probabilistic, 1 worst case
  // worst case: |dz_k| <= delta_per_norm * n for every k
  float delta_per_norm;
  float delta_abs;        // FP16: the subnormal halves' absolute part of |dz_k|
  float rel;              // relative bound of the reductions of sum g
  float sum_w;            // sum of the elliptic weights
  // probabilistic: lambda * sqrt(s_rep^2 + s_acc^2 + s_eval^2) + bias + quad
  float lambda;           // margin in standard deviations
  float rep_k, rep_f;     // per-entry residual scale rep = rep_k max_j |a_j| + rep_f (u_s^2, FP16 floors);
                          // s_rep = sqrt(3) rep H
  float acc_c;            // s_acc = acc_c * n * H (accumulation roundings of both products)
  float eval_c;           // g evaluations: eval_c * |f|
  float sum_u, sum_f2, sum_t2;   // sums over k: sum_u * sqrt(sum_f2 f^2 + sum_t2 sum_c T'_c^2)
  float quad_a, quad_b;   // second-order term quad_a rep^2 + quad_b n^2
  float bias_c;           // mean truncation of the leading product: bias_c * sum_k |g'(z_k)| |z_k|
                          // (n H Rastrigin, 2|f| elliptic)
  float bias_c2;          // truncation bias of the two correction products (and the subnormal
                          // halves' absolute part): bias_c2 * n * H
  float hconst;           // Rastrigin: 20 pi sqrt(D)
  float wmax;             // elliptic: the largest weight
};

// The elliptic weight of column k: 10^(6k/(D-1)) = 2^(k * ell_k).
__device__ __forceinline__ float sr_weight(int obj, int k, float ell_k) {
  return obj == kSrElliptic ? exp2f((float)k * ell_k) : 1.0f;
}

__device__ __forceinline__ float sr_g(int obj, float z, float w) {
  return obj == kSrElliptic ? w * z * z : fmaf(z, z, 20.0f * sin2pi(z));
}

// Asynchronous global -> shared copies (LDGSTS) of 16 or 4 bytes; src_bytes = 0
// fills the destination with zeros and reads nothing.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ uint32_t sr_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

}  // namespace de
