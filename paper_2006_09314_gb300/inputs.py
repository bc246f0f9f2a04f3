"""Seeded synthetic inputs for the control equation (A^-alpha + beta A^alpha) u = y_Omega.

This module only *samples* problem data: the three separable coefficient
functions a_l at the half-points of the grid, and the canonical factors of the
design function y_Omega. It contains none of the method's arithmetic (no
operator assembly, no eigendecomposition, no spectral function), so both the
CPU oracle and the GPU library can be fed from it without sharing any of the
computation they are compared on.

Problem family (the paper's setting, Section 2 and Section 3.2):
  * domain (0,1)^3, n interior finite-difference points per axis,
    h = 1/(n+1), x_i = i*h;
  * diagonal separable coefficient diag{a_1(x_1), a_2(x_2), a_3(x_3)} with
    a_l(x) = 1 + 0.5*sin(pi*x + phi_l), phi_l ~ U[0, pi), sampled at the
    half-points x_{i-1/2} = (i - 1/2)*h, i = 1..n+1 (range [0.5, 1.5], so the
    operator is uniformly elliptic);
  * design function y_Omega in canonical format (Appendix 1, "CP_form") with
    unit weights; every factor is a sum of three sines sin(k*pi*x) with
    distinct k drawn from {1..5} and N(0,1) amplitudes.

The paper's own design functions ("box" and "H" shapes, Section 4) appear only
as figures without formulas, so these seeded sine factors stand in for them.
Seeds follow seed = 1000*config_id + problem_index.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "make_problem",
    "coefficient_half_points",
    "sine_factors",
    "CONFIGS",
    "problem_seed",
    "batch_problems",
]


def problem_seed(config_id: int, index: int) -> int:
    """Seed of problem `index` of configuration `config_id`."""
    return 1000 * int(config_id) + int(index)


@dataclasses.dataclass
class Problem:
    """One seeded control problem (inputs only).

    coeffs : (3, n+1) float64, a_l(x_{i-1/2}) for i = 1..n+1 (row l = mode l).
    yw     : (S,) float64, canonical weights of y_Omega (all ones).
    yU     : list of three (n, S) float64 arrays, column j = factor of term j
             in mode l, sampled at x_i = i*h, i = 1..n.
    """

    n: int
    alpha: float
    beta: float
    coeffs: np.ndarray
    yw: np.ndarray
    yU: list
    phis: np.ndarray
    seed: int


def coefficient_half_points(n: int, phi: float) -> np.ndarray:
    """a(x) = 1 + 0.5 sin(pi x + phi) at x_{i-1/2} = (i-1/2)/(n+1), i=1..n+1."""
    h = 1.0 / (n + 1)
    xh = (np.arange(1, n + 2, dtype=np.float64) - 0.5) * h
    return 1.0 + 0.5 * np.sin(np.pi * xh + phi)


def sine_factors(n: int, rank: int, rng: np.random.Generator) -> np.ndarray:
    """(n, rank) matrix; column j = sum over 3 distinct k in {1..5} of c_k sin(k pi x_i)."""
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1, dtype=np.float64) * h
    out = np.empty((n, rank), dtype=np.float64)
    for j in range(rank):
        ks = rng.choice(np.arange(1, 6), size=3, replace=False)
        cs = rng.standard_normal(3)
        col = np.zeros(n)
        for k, c in zip(ks, cs):
            col += c * np.sin(k * math.pi * x)
        out[:, j] = col
    return out


def make_problem(n: int, alpha: float, beta: float, rank: int, seed: int) -> Problem:
    """Seeded problem: coefficients first (3 phases), then the 3 factor matrices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    phis = rng.uniform(0.0, math.pi, size=3)
    coeffs = np.stack([coefficient_half_points(n, p) for p in phis])
    yU = [sine_factors(n, rank, rng) for _ in range(3)]
    yw = np.ones(rank, dtype=np.float64)
    return Problem(n=n, alpha=float(alpha), beta=float(beta), coeffs=coeffs,
                   yw=yw, yU=yU, phis=phis, seed=seed)


# Workload configurations (sizes of the paper's 3D experiments, Section 4.2,
# n = 64..512, and rank-structured grids up to 2048).
CONFIGS = {
    # small case: n = 32, alpha = 0.5, beta = 1e-2, design rank 3, eps = 1e-6
    0: dict(n=[32], alpha=[0.5], beta=[1e-2], rank=3, eps=1e-6),
    # at scale: rank-structured n in {256..2048}, 3 alphas x 3 betas, rank 5
    1: dict(n=[256, 512, 1024, 2048], alpha=[0.25, 0.5, 0.75],
            beta=[1e-4, 1e-2, 1.0], rank=5, eps=1e-6,
            fullgrid_n=[128, 256, 512]),
    # precision: full grid n = 512 and rank-structured n = 2048
    2: dict(n=[512, 2048], alpha=[0.5], beta=[1e-2], rank=5, eps=1e-6),
}


def batch_problems(count: int, seed: int, n_choices=tuple(range(64, 513, 32))):
    """Uneven batch (f-2 workload): n uniform in n_choices, design rank uniform in
    1..8, alpha ~ U[0.2, 0.8], log10 beta ~ U[-4, 0]; problem i from seed + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.choice(n_choices))
        rank = int(rng.integers(1, 9))
        alpha = float(rng.uniform(0.2, 0.8))
        beta = float(10.0 ** rng.uniform(-4.0, 0.0))
        out.append(make_problem(n, alpha, beta, rank, seed + 1 + i))
    return out
