"""Seeded synthetic inputs for the DE generation step.

This module holds the workload definitions and the seeded generators that
both the CUDA path and its CPU checker consume: parent populations, the shift
vector and rotation matrix of the shifted-rotated objectives, and the
instance list of the batched workload. It holds none of the method's
arithmetic (no draws, mutation, crossover, fitness or selection).

The paper uses closed-form test functions only (Section 4: Ackley,
Griewank, Rosenbrock), so every workload here is synthetic by nature.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Search boxes per objective. Ackley, Griewank and Rosenbrock as given in
# Section 4; sphere, Rastrigin and elliptic use their textbook boxes; the
# shifted-rotated forms use [-100, 100] so that a shift drawn from
# [-80, 80] keeps the optimum inside the box.
BOXES = {
    "sphere": (-100.0, 100.0),
    "rastrigin": (-5.12, 5.12),
    "ackley": (-30.0, 30.0),
    "rosenbrock": (-5.12, 5.12),
    "griewank": (-400.0, 400.0),
    "elliptic": (-100.0, 100.0),
    "sr_rastrigin": (-100.0, 100.0),
    "sr_elliptic": (-100.0, 100.0),
}


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    D: int
    objective: str
    crossovers: tuple
    F: float
    CRs: tuple
    generations: int
    seed: int
    notes: str = ""
    objectives: tuple = field(default=())

    @property
    def box(self):
        return BOXES[self.objective]


# The five synthetic workloads (sizes of the large-scale runs the method is
# aimed at; Tables II-V use the same functions at D = 50 .. 1000).
SPHERE_N100_D30 = Workload("sphere_N100_D30", 100, 30, "sphere", ("exp", "nec", "bin"),
                           0.5, (0.9,), 200, 1)
RASTRIGIN_N1024_D1000 = Workload("rastrigin_N1024_D1000", 1024, 1000, "rastrigin",
                                 ("bin", "exp", "nec"), 0.5, (0.1, 0.5, 0.9), 1000, 1)
SR_N4096_D1024 = Workload("shifted_rotated_N4096_D1024", 4096, 1024, "sr_rastrigin",
                          ("nec",), 0.5, (0.9,), 1000, 1,
                          objectives=("sr_rastrigin", "sr_elliptic"))
BATCHED_512 = Workload("batched_512_instances", 0, 0, "sphere", ("nec",), 0.5, (0.9,), 500, 4,
                       objectives=("sphere", "rastrigin", "ackley", "rosenbrock"))
LARGEST_N16384_D10000 = Workload("rosenbrock_ackley_N16384_D10000", 16384, 10000, "rosenbrock",
                                 ("nec", "bin", "exp"), 0.5, (0.9,), 100, 1,
                                 objectives=("rosenbrock", "ackley"))

ALL = (SPHERE_N100_D30, RASTRIGIN_N1024_D1000, SR_N4096_D1024, BATCHED_512,
       LARGEST_N16384_D10000)


def population(N: int, D: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """A uniform N x D float32 population in [lo, hi] (numpy PCG64 stream)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(N, D)).astype(np.float32)
    return np.clip(x, np.float32(lo), np.float32(hi))


def shift_vector(D: int, seed: int = 2, lo: float = -80.0, hi: float = 80.0) -> np.ndarray:
    """Shift o ~ U[lo, hi]^D as float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=D).astype(np.float32)


def rotation(D: int, seed: int = 3, dtype=np.float32) -> np.ndarray:
    """Q of the QR factorisation of a seeded D x D Gaussian matrix, with the
    column signs fixed by sign(diag R) so that Q is unique (FP64 QR, then cast)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((D, D))
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    q = q * s[None, :]
    return q.astype(dtype)


@dataclass(frozen=True)
class InstanceSpec:
    N: int
    D: int
    objective: str


def batched_specs(n_inst: int = 512, seed: int = 4, d_lo: int = 10, d_hi: int = 2000,
                  n_cap: int = 4096) -> list:
    """Instances of the batched workload: D log-uniform in [d_lo, d_hi]
    (rounded), N = min(10 D, n_cap), objectives assigned round-robin over
    sphere, Rastrigin, Ackley, Rosenbrock."""
    rng = np.random.default_rng(seed)
    Ds = np.round(np.exp(rng.uniform(math.log(d_lo), math.log(d_hi), size=n_inst))).astype(int)
    objs = BATCHED_512.objectives
    return [InstanceSpec(int(min(10 * d, n_cap)), int(d), objs[k % len(objs)])
            for k, d in enumerate(Ds)]
