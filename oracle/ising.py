"""Ising site tensor T0 (SM Sec. A: Z = sum over spins of a product of local
rank-4 tensors built from Boltzmann weights).

Reading used (the paper's SM Sec. A draws a plaquette tensor; the
coarse-graining count "2^n sites after n steps" needs one tensor per spin):
one tensor per spin, H = -J sum_<ij> s_i s_j - h sum_i s_i, s = +-1.  Each
bond weight exp(beta J s s') is split symmetrically as W W^T with

    W[s, 0] = sqrt(cosh(beta J)),   W[s, 1] = s * sqrt(sinh(beta J)),

so that sum_b W[s, b] W[s', b] = cosh + s s' sinh = exp(beta J s s').  The
site tensor carries the spin sum and the field weight:

    T0[l, r, u, d] = sum_s exp(beta h s) W[s, l] W[s, r] W[s, u] W[s, d].

Requires beta * J >= 0 (the square-root split needs sinh(beta J) >= 0).
Spin index 0 is s = +1, index 1 is s = -1.
"""
from __future__ import annotations

import math

import numpy as np

_SPINS = (1.0, -1.0)


def _bond_factor(beta: float, J: float):
    k = beta * J
    if k < 0:
        raise ValueError("oracle Ising tensor needs beta*J >= 0")
    return math.sqrt(math.cosh(k)), math.sqrt(math.sinh(k))


def ising_T0(beta: float, J: float = 1.0, h: float = 0.0) -> np.ndarray:
    """Rank-4 site tensor T0[l, r, u, d] of shape (2, 2, 2, 2), float64."""
    a, b = _bond_factor(beta, J)
    T = np.zeros((2, 2, 2, 2))
    for s in _SPINS:
        W = np.array([a, s * b])
        T += math.exp(beta * h * s) * np.einsum("l,r,u,d->lrud", W, W, W, W)
    return T


def ising_dT0_dbeta(beta: float, J: float = 1.0, h: float = 0.0) -> np.ndarray:
    """Analytic d T0 / d beta (product rule over the five beta-dependent
    factors exp(beta h s), W[s,l], W[s,r], W[s,u], W[s,d]).  Needs beta J > 0
    when J != 0 (the derivative of sqrt(sinh) diverges at 0)."""
    k = beta * J
    a, b = _bond_factor(beta, J)
    ch, sh = math.cosh(k), math.sinh(k)
    da = J * sh / (2.0 * a)                       # d sqrt(cosh k) / d beta
    db = J * ch / (2.0 * b) if b > 0 else 0.0     # d sqrt(sinh k) / d beta
    dT = np.zeros((2, 2, 2, 2))
    for s in _SPINS:
        e = math.exp(beta * h * s)
        de = h * s * e
        W = np.array([a, s * b])
        dW = np.array([da, s * db])
        dT += de * np.einsum("l,r,u,d->lrud", W, W, W, W)
        dT += e * (np.einsum("l,r,u,d->lrud", dW, W, W, W)
                   + np.einsum("l,r,u,d->lrud", W, dW, W, W)
                   + np.einsum("l,r,u,d->lrud", W, W, dW, W)
                   + np.einsum("l,r,u,d->lrud", W, W, W, dW))
    return dT
