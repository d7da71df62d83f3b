"""Scheme (b) of differentiable TRG on the GPU: exponential cooling of the
quantum XY chain's density matrix (main text Fig. 1b and the XY-chain
paragraph; SM Sec. F for rho(tau)).

One vertical merge is the MPO product rho(2 tau) = rho(tau) rho(tau) with the
doubled bond compressed by an isometry; the depth-k chain is evaluated as
Tr[rho rho] on the infinite chain (the exact final product), i.e. at
beta = 2^(k+1) tau.  With n_d > 0 the isometries of the last n_d layers are
optimised after every step by MERA updates against that free energy
(differentiable TRG, main text Eq. (1) and the MERA paragraph).

Everything runs through the C ABI (forward_xy, backward, mera_update,
set_given_steps); this module only drives the loop and converts the
per-copy value to per-site thermodynamics.
"""
from __future__ import annotations

import numpy as np

from . import Plan


def per_site(lnz_per_copy: np.ndarray, depths: np.ndarray, tau: float):
    """(beta_k, ln Z / N per site, f per site) at depth k: beta = 2^(k+1) tau,
    ln Z per two-site cell = 2^(k+1) lnz."""
    depths = np.asarray(depths, dtype=np.float64)
    beta = tau * 2.0 ** (depths + 1)
    lnz_site = 2.0 ** depths * np.asarray(lnz_per_copy)
    return beta, lnz_site, -lnz_site / beta


def cooling(tau: float, d_cut: int, n_steps: int, J: float = 1.0, n_d: int = 0,
            n_sweeps: int = 1, n_inner: int = 5, **plan_kw) -> dict:
    """Cool from rho(tau) through n_steps doublings.  n_d = 0: plain scheme (b)
    (isometries from the local HOSVD, one forward); n_d >= 1: after each new
    layer the last n_d layers get n_sweeps sweeps of n_inner MERA updates.

    Returns dict(beta, lnz_site, f, lnz_copy) over depths 1..n_steps."""
    depths = np.arange(1, n_steps + 1)
    if n_d <= 0:
        with Plan(4, d_cut, n_steps, want_grad=False, scheme=1, chain_steps=True,
                  **plan_kw) as p:
            p.forward_xy(tau, J)
            lnz = p.chain_lnz_steps()
    else:
        lnz = np.zeros(n_steps)
        with Plan(4, d_cut, n_steps, want_grad=True, fixed_w_grad=True, w_given=True,
                  scheme=1, **plan_kw) as p:
            for k in depths:
                p.set_steps(k)
                p.set_given_steps(k - 1)
                p.forward_xy(tau, J)             # layer k from its local HOSVD
                p.set_given_steps(k)
                for _ in range(n_sweeps):
                    for layer in range(max(1, k - n_d + 1), k + 1):
                        for _ in range(n_inner):
                            p.forward_xy(tau, J)
                            p.backward()
                            p.mera_update(layer)
                lnz[k - 1] = p.forward_xy(tau, J)[0]
    beta, lnz_site, f = per_site(lnz, depths, tau)
    return dict(beta=beta, lnz_site=lnz_site, f=f, lnz_copy=lnz)
