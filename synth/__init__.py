"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws and shapes inputs; it holds none of the HOTRG
arithmetic (no site tensor from Boltzmann weights, no contraction, no
eigendecomposition).  Both the oracle and the CUDA path receive what is
generated here as plain arrays or scalars.

Workloads (the paper studies the square-lattice Ising model, main text
"dTRG of 2D Ising model" and SM Sec. A; there is no dataset, so every
input is synthetic):

* ``beta_grid``: 64 inverse temperatures on [0.30, 0.60] (both ends
  included), J = 1, h = 0 -- a dense temperature scan across the critical
  point, the analogue of the paper's temperature sweeps.
* ``random_symmetric_T0``: a random rank-4 tensor of bond dimension d0,
  entries N(0, 1), made symmetric under the lattice reflections l<->r and
  u<->d by averaging the four reflected copies, then scaled so that
  max|T| = 1.
* ``random_T0``: the same draw without the symmetrisation (a tensor whose
  left and right environments differ).
* ``serving_stream``: a seeded Poisson stream of Ising solve requests.
"""
from __future__ import annotations

import math

import numpy as np

BETA_C = 0.5 * math.log1p(math.sqrt(2.0))  # Ising critical point for J = 1


def beta_grid(n: int = 64, lo: float = 0.30, hi: float = 0.60) -> np.ndarray:
    """``n`` equally spaced inverse temperatures on [lo, hi], ends included."""
    return np.linspace(lo, hi, n)


def random_symmetric_T0(seed: int, d0: int = 4) -> np.ndarray:
    """Random reflection-symmetric rank-4 tensor T[l, r, u, d], max|T| = 1.

    Entries are ``default_rng(seed).standard_normal(d0**4)`` reshaped to
    (l, r, u, d); the tensor is then averaged over the identity, the l<->r
    swap, the u<->d swap and both swaps, and divided by its largest
    magnitude.  Returned as a C-contiguous float64 array.
    """
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(d0 ** 4).reshape(d0, d0, d0, d0)
    t = 0.25 * (t + t.transpose(1, 0, 2, 3) + t.transpose(0, 1, 3, 2)
                + t.transpose(1, 0, 3, 2))
    t = t / np.abs(t).max()
    return np.ascontiguousarray(t, dtype=np.float64)


def random_T0(seed: int, d0: int = 4) -> np.ndarray:
    """Random rank-4 tensor T[l, r, u, d] with N(0, 1) entries
    (``default_rng(seed)``), divided by its largest magnitude."""
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(d0 ** 4).reshape(d0, d0, d0, d0)
    return np.ascontiguousarray(t / np.abs(t).max(), dtype=np.float64)


def serving_stream(seed: int = 2024, n: int = 10000, rate: float = 200.0,
                   d_cuts=(16, 24, 32, 48, 64), steps=(20, 40),
                   beta_range=(0.30, 0.60), h_range=(0.0, 0.05),
                   p_grad: float = 0.5):
    """Seeded Poisson stream of Ising solve requests.

    Returns a list of dicts with keys ``t_arrival`` (seconds from start),
    ``beta``, ``J`` (= 1), ``h``, ``d_cut``, ``n_steps``, ``want_grad``.
    Inter-arrival times are exponential with mean 1/rate; beta and h are
    uniform on their ranges, d_cut uniform over ``d_cuts``, n_steps uniform
    on the inclusive integer range ``steps``, want_grad Bernoulli(p_grad).
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    beta = rng.uniform(beta_range[0], beta_range[1], size=n)
    h = rng.uniform(h_range[0], h_range[1], size=n)
    dc = rng.choice(np.asarray(d_cuts), size=n)
    ns = rng.integers(steps[0], steps[1] + 1, size=n)
    g = rng.random(n) < p_grad
    return [dict(t_arrival=float(t[i]), beta=float(beta[i]), J=1.0, h=float(h[i]),
                 d_cut=int(dc[i]), n_steps=int(ns[i]), want_grad=bool(g[i]))
            for i in range(n)]
