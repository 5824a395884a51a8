"""Seeded synthetic inputs for the Laplace KIFMM workloads.

This module only draws random numbers; it holds none of the method's
arithmetic.  Both the CPU oracle tests and the CUDA path take their inputs
from here, so the two sides always see identical points and charges.

The paper evaluates on random point clouds (random points on the surface of
a sphere, "Parallelization strategies for FMM operators" section); it uses no
public dataset.  Every generator uses numpy's PCG64 (``default_rng(seed)``)
and draws the points first, then the charges.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def uniform_cube(n: int, seed: int, nrhs: int = 1):
    """n points uniform in [0,1]^3, charges uniform in [-1,1] (n, nrhs)."""
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3))
    q = rng.uniform(-1.0, 1.0, size=(n, nrhs))
    return x, q


def sphere_surface(n: int, seed: int, nrhs: int = 1):
    """n points uniform on the unit sphere (normalised Gaussian vectors),
    charges N(0,1) (n, nrhs)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    x = g / np.linalg.norm(g, axis=1, keepdims=True)
    q = rng.standard_normal((n, nrhs))
    return x, q


def gaussian_mixture(n: int, seed: int, nrhs: int = 1, clusters: int = 8,
                     sigma: float = 0.05):
    """n points from an equal-weight mixture of isotropic Gaussians with
    centres uniform in [0,1]^3 and standard deviation sigma (not clipped);
    charges uniform in [-1,1] (n, nrhs)."""
    rng = np.random.default_rng(seed)
    centres = rng.random((clusters, 3))
    which = rng.integers(0, clusters, size=n)
    x = centres[which] + sigma * rng.standard_normal((n, 3))
    q = rng.uniform(-1.0, 1.0, size=(n, nrhs))
    return x, q


def log_uniform_sizes(count: int, seed: int, lo: float = 1e3, hi: float = 1e5):
    """Problem sizes N_i = round(10^U[log10 lo, log10 hi])."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(math.log10(lo), math.log10(hi), size=count)
    return np.rint(10.0 ** e).astype(np.int64)


def batch_problems(count: int, seed: int, nrhs: int = 1, lo: float = 1e3, hi: float = 1e5):
    """`count` independent problems, N_i log-uniform in [lo, hi], each N_i
    points uniform in [0,1]^3 with charges uniform in [-1,1]; list of
    (x_i, q_i)."""
    sizes = log_uniform_sizes(count, seed, lo, hi)
    return [uniform_cube(int(n), 1_000_000 * (seed + 1) + i, nrhs) for i, n in enumerate(sizes)]


def sample_targets(n: int, m: int, seed: int):
    """m distinct target indices out of n (sorted), for sampled error checks."""
    rng = np.random.default_rng(seed + 1_000_003)
    m = min(m, n)
    return np.sort(rng.choice(n, size=m, replace=False))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: point distribution, size and FMM parameters.
    kind "batch": `problems` independent uniform cubes of log-uniform sizes
    (batch_problems), evaluated as one plan; n is their total at seed 0 and
    error_samples the sampled targets per problem."""
    name: str
    kind: str            # "cube" | "sphere" | "gauss" | "batch"
    n: int
    p: int
    ncrit: int
    nrhs: int = 1
    error_samples: int = 0   # 0: all targets
    problems: int = 0

    def problem_sets(self, seed: int = 0):
        """kind "batch": the list of (x_i, q_i)."""
        return batch_problems(self.problems, seed, self.nrhs)

    def generate(self, seed: int = 0):
        if self.kind == "batch":
            sets = self.problem_sets(seed)
            return (np.concatenate([x for x, _ in sets]),
                    np.concatenate([q for _, q in sets]))
        gen = {"cube": uniform_cube, "sphere": sphere_surface,
               "gauss": gaussian_mixture}[self.kind]
        return gen(self.n, seed, self.nrhs)


# The five workloads of the hot-path study, by what they are.
CUBE_10K_P4 = Workload("cube_n1e4_p4_ncrit64", "cube", 10_000, 4, 64)
CUBE_1M_P6 = Workload("cube_n1e6_p6_ncrit150", "cube", 1_000_000, 6, 150,
                      error_samples=1000)
SPHERE_4M_P7 = Workload("sphere_n4e6_p7_ncrit128", "sphere", 4_000_000, 7, 128,
                        error_samples=1000)
CUBE_1M_P6_NRHS64 = Workload("cube_n1e6_p6_ncrit150_nrhs64", "cube", 1_000_000,
                             6, 150, nrhs=64, error_samples=1000)
GAUSS_16M_P8 = Workload("gauss8_n1.6e7_p8_ncrit128_nrhs8", "gauss", 16_000_000,
                        8, 128, nrhs=8, error_samples=2000)

BATCH_256_P6 = Workload("batch256_cube_p6_ncrit150", "batch",
                        int(log_uniform_sizes(256, 0).sum()), 6, 150,
                        error_samples=8, problems=256)

WORKLOADS = {w.name: w for w in
             (CUBE_10K_P4, CUBE_1M_P6, SPHERE_4M_P7, CUBE_1M_P6_NRHS64,
              GAUSS_16M_P8, BATCH_256_P6)}
