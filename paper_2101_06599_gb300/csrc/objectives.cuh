// objectives.cuh — FP32 row fitness as per-gene partial sums plus a final
// combine, written in cancellation-free forms so that the FP32 value stays
// within 1e-5 max(1, |f|) of the exact value near the optima:
//
//  sphere      sum x^2
//  Rastrigin   10 D + sum (x^2 - 10 cos 2 pi x) = sum (x^2 + 20 sin^2(pi x))
//  Ackley      (Section 4) -20 exp(-b sqrt(m2)) - exp(mc) + 20 + e with
//              m2 = mean x^2 and mc = mean cos 2 pi x = 1 - 2 mean sin^2(pi x):
//              f = -20 expm1(-b sqrt(m2)) - e expm1(-2 mean sin^2(pi x))
//  Rosenbrock  (Section 4) sum_{j<D-1} 100 (x_j^2 - x_{j+1})^2 + (1 - x_j)^2,
//              with x_j^2 - x_{j+1} as one fused multiply-add
//  Griewank    (Section 4) sum x^2 / 4000 - prod cos(x_j / sqrt(j+1)) + 1;
//              the product is carried as sum log|cos| plus a sign count,
//              log cos y = log1p(-2 sin^2(y/2)) while cos y > 1/2, and
//              1 - prod = -expm1(sum log cos) when the sign is positive
//  elliptic    sum 10^(6 j / (D-1)) x_j^2 = sum 2^(j * 6 log2(10) / (D-1)) x_j^2
#pragma once
#include "common.cuh"

namespace de {

// sin^2(pi x) = r^2 Q(r^2), r = x - rint(x) (exact), Q a degree-5 fit of
// sin^2(pi sqrt t) / t on t in [0, 1/4]; coefficients from sin2pi_poly.py
// (relative error of the fit 1.4e-8, of the FP32 evaluation ~2e-7).
__device__ __forceinline__ float sin2pi(float x) {
  const float r = x - rintf(x);
  const float t = r * r;
  float q = -3.335728645e+00f;
  q = fmaf(q, t, 1.303679657e+01f);
  q = fmaf(q, t, -3.009848022e+01f);
  q = fmaf(q, t, 4.272692108e+01f);
  q = fmaf(q, t, -3.246966171e+01f);
  q = fmaf(q, t, 9.869604111e+00f);
  return q * t;
}

struct Acc {
  float a, b, c;   // partial sums (meaning depends on the objective)
};

template <int OBJ> struct ObjTraits { static constexpr int kSums = 1; };
template <> struct ObjTraits<kAckley> { static constexpr int kSums = 2; };
template <> struct ObjTraits<kGriewank> { static constexpr int kSums = 3; };

// One gene j with value x (not used for Rosenbrock, which takes pairs).
template <int OBJ>
__device__ __forceinline__ void accum_gene(Acc& s, float x, int j, const GenParams& p) {
  if constexpr (OBJ == kSphere) {
    s.a = fmaf(x, x, s.a);
  } else if constexpr (OBJ == kRastrigin) {
    s.a += fmaf(x, x, 20.0f * sin2pi(x));
  } else if constexpr (OBJ == kAckley) {
    s.a = fmaf(x, x, s.a);
    s.b += sin2pi(x);
  } else if constexpr (OBJ == kGriewank) {
    s.a = fmaf(x, x, s.a);
    const float y = x * rsqrtf((float)(j + 1));
    const float h = sinf(0.5f * y);
    const float c = fmaf(-2.0f * h, h, 1.0f);          // cos y = 1 - 2 sin^2(y/2)
    s.b += (c > 0.5f) ? log1pf(-2.0f * h * h) : logf(fabsf(c));
    s.c += (c < 0.0f) ? 1.0f : 0.0f;
  } else if constexpr (OBJ == kElliptic) {
    const float w = exp2f((float)j * p.ell_k);
    s.a = fmaf(w * x, x, s.a);
  }
}

// Rosenbrock term of the pair (x_j, x_{j+1}).
__device__ __forceinline__ void accum_pair(Acc& s, float x, float xn) {
  const float d = fmaf(x, x, -xn);
  const float e = 1.0f - x;
  s.a += fmaf(100.0f * d, d, e * e);
}

// Row value from the reduced sums.
template <int OBJ>
__device__ __forceinline__ float finalize_fitness(const Acc& s, const GenParams& p) {
  if constexpr (OBJ == kAckley) {
    const float invD = 1.0f / (float)p.D;
    const float t1 = -20.0f * expm1f(-p.ackley_b * sqrtf(s.a * invD));
    const float t2 = -2.71828182845904523536f * expm1f(-2.0f * s.b * invD);
    return t1 + t2;
  } else if constexpr (OBJ == kGriewank) {
    const bool neg = (((int)s.c) & 1) != 0;
    const float one_minus_prod = neg ? 1.0f + expf(s.b) : -expm1f(s.b);
    return fmaf(s.a, 1.0f / 4000.0f, one_minus_prod);
  } else {
    return s.a;
  }
}

}  // namespace de
