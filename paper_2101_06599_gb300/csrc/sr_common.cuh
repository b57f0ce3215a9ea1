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

constexpr int kSrTile = 64;          // FP32 GEMM: 64 x 64 output tile
constexpr int kSrKStep = 32;         // FP32 GEMM: K per shared-memory stage

struct SrParams {
  GenParams g;
  int obj;                 // kSrRastrigin or kSrElliptic
  int prec;                // 0 = FP32, 2 = BF16 (split hi/lo operands)
  int nct;                 // column tiles per row of part_g / part_w (the main product)
  int nct2;                // column tiles per entry of part2_g / part2_w (FP32 product)
  const float* shift;      // o, D floats
  const float* rot;        // R, D x D FP32 row-major (z_k = sum_j R[k][j] a_j)
  const uint16_t* rot_hi;  // bf16(R), D x D
  const uint16_t* rot_lo;  // bf16(R - bf16(R)), D x D
  uint16_t* a_hi;          // bf16(u - o), N x D (BF16 path)
  uint16_t* a_lo;          // bf16((u - o) - bf16(u - o)), N x D
  float* part_g;           // N x nct: sum of g(z) over the column tile
  float* part_w;           // N x nct: sum of w_k |z_k| (w = 1 Rastrigin, c_k elliptic)
  float* norm2;            // N: |u - o|^2 of the trial (FP32)
  float* fit_err;          // N: bound on |fit - FP32-path value| of the stored parent
  int* amb;                // ambiguous entries: row << 1 | (1 = parent row)
  unsigned* amb_count;     // number of entries in amb
  float* part2_g;          // 2N x nct: partial sums of the re-evaluated entries
  float* part2_w;
};

// Bound constants of the BF16 path (sr_select_kernel).
struct SrBound {
  float delta_per_norm;   // per-element |dz| bound per unit |u - o|_2
  float rel;              // relative bound of the reductions of sum g
  float sum_w;            // sum of the elliptic weights
};

// The elliptic weight of column k: 10^(6k/(D-1)) = 2^(k * ell_k).
__device__ __forceinline__ float sr_weight(int obj, int k, float ell_k) {
  return obj == kSrElliptic ? exp2f((float)k * ell_k) : 1.0f;
}

__device__ __forceinline__ float sr_g(int obj, float z, float w) {
  return obj == kSrElliptic ? w * z * z : fmaf(z, z, 20.0f * sin2pi(z));
}

}  // namespace de
