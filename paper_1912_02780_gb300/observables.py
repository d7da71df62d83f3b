"""Thermodynamics of the square-lattice Ising model from HOTRG solves.

For each inverse temperature beta on a grid the library returns ln Z / N and,
from the hand-written backward, d(ln Z / N)/d beta.  From these:

    f(beta) = -ln Z / (N beta)                      free energy per site
    u(beta) = -d(ln Z / N)/d beta                    internal energy per site
    c(beta) = beta^2 d^2(ln Z / N)/d beta^2 = -beta^2 du/dbeta

The paper obtains such derivatives numerically (main text, energy as the
derivative of beta f); here u comes from the adjoint and c from a
second-order finite difference of u on the grid (central inside, one-sided
at the two ends), the same rule the oracle applies to its own u.
"""
from __future__ import annotations

import numpy as np

from . import Plan


def grid_derivative(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Second-order finite-difference dy/dx on a uniform grid (central inside,
    one-sided three-point at the ends)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    h = x[1] - x[0]
    d = np.empty_like(y)
    d[1:-1] = (y[2:] - y[:-2]) / (2 * h)
    d[0] = (-3 * y[0] + 4 * y[1] - y[2]) / (2 * h)
    d[-1] = (3 * y[-1] - 4 * y[-2] + y[-3]) / (2 * h)
    return d


def ising_thermodynamics(betas, d_cut: int, n_steps: int, precision: str = "fp64",
                         split_from_step: int = 1, J: float = 1.0, h: float = 0.0,
                         hi_precision_steps: int = 2) -> dict:
    """ln Z / N, f, u and c on a beta grid (one plan reused for every beta)."""
    betas = np.asarray(betas, dtype=np.float64)
    lnz = np.empty_like(betas)
    dlnz = np.empty_like(betas)
    with Plan(2, d_cut, n_steps, precision, split_from_step=split_from_step, want_grad=True,
              hi_precision_steps=hi_precision_steps) as p:
        for i, b in enumerate(betas):
            lnz[i], _, _ = p.forward_ising(float(b), J, h)
            _, dlnz[i] = p.backward(want_dbeta=True)
    u = -dlnz
    c = -betas ** 2 * grid_derivative(betas, u) if len(betas) >= 3 else np.full_like(betas, np.nan)
    return dict(beta=betas, lnz=lnz, f=-lnz / betas, u=u, c=c)
