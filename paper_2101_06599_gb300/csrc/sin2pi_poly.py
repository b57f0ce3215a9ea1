"""Coefficients of the sin^2(pi x) approximation used by the Rastrigin and
Ackley objectives (objectives.cuh), derived here from the mathematics.

For r = x - rint(x) in [-1/2, 1/2] (exact in FP32), sin^2(pi x) = sin^2(pi r)
= r^2 Q(r^2) with Q(t) = sin^2(pi sqrt t) / t, analytic on t in [0, 1/4]
(Q(0) = pi^2, Q(1/4) = 4). Q is fitted by a degree-5 polynomial with weighted
least squares at Chebyshev nodes (weight 1/Q: relative error), in FP64.

Run: python sin2pi_poly.py  -> prints the coefficients (highest degree first)
and the maximum relative error of the FP64 fit and of an FP32 Horner
evaluation over a dense grid.
"""
import numpy as np

DEG = 5


def q_exact(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    small = t < 1e-12
    out[small] = np.pi ** 2 - np.pi ** 4 * t[small] / 3.0
    tt = t[~small]
    out[~small] = np.sin(np.pi * np.sqrt(tt)) ** 2 / tt
    return out


def fit(deg=DEG, nodes=400):
    k = np.arange(nodes)
    t = 0.125 + 0.125 * np.cos(np.pi * (k + 0.5) / nodes)      # Chebyshev nodes on [0, 1/4]
    y = q_exact(t)
    A = np.vander(t, deg + 1) / y[:, None]
    c, *_ = np.linalg.lstsq(A, np.ones_like(t), rcond=None)
    return c                                                     # highest degree first


def check(c):
    r = np.linspace(-0.5, 0.5, 2_000_001)
    truth = np.sin(np.pi * r) ** 2
    t = r * r
    p64 = np.polyval(c, t) * t
    nz = truth > 1e-30
    e64 = np.max(np.abs(p64[nz] - truth[nz]) / truth[nz])
    r32 = r.astype(np.float32)
    t32 = r32 * r32
    acc = np.float32(c[0])
    for ci in c[1:]:
        acc = acc * t32 + np.float32(ci)                          # FP32 Horner (FMA-free bound)
    p32 = (acc * t32).astype(np.float64)
    truth32 = np.sin(np.pi * r32.astype(np.float64)) ** 2
    nz = truth32 > 1e-30
    e32 = np.max(np.abs(p32[nz] - truth32[nz]) / truth32[nz])
    return e64, e32


if __name__ == "__main__":
    c = fit()
    e64, e32 = check(c)
    for ci in c:
        print("%.9e" % np.float32(ci))
    print("max relative error: fit %.3e, fp32 horner %.3e" % (e64, e32))
