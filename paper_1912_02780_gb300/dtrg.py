"""Differentiable-TRG sweeps on the GPU (main text: second renormalization as
backpropagation, Eq. (1), and the MERA update of the isometries).

HOTRG fixes each isometry w_k from the leading eigenvectors of its Gram
matrix.  Differentiable TRG treats the w_k as parameters: one backward with
every w held fixed gives the environment E_w = d(ln Z/N)/d w_k of each one,
and the MERA update replaces w_k by the polar factor U V^T of E_w = U S V^T,
the isometry maximising Tr(E_w^T w).  A sweep updates k = 1..n (the first
coarse-graining step is the innermost layer), each n_inner times with a fresh
environment; the sweep starts from the HOTRG isometries.

Everything runs through the C ABI (forward, backward, hotrg_mera_update: the
cuSOLVER SVD and the FP64 GEMM forming U V^T); this module only drives the
loop.
"""
from __future__ import annotations

import numpy as np

from . import LBFGS, Plan


def dtrg_sweeps(d0: int, d_cut: int, n_steps: int, n_sweeps: int, n_inner: int = 1,
                T0=None, beta: float | None = None, J: float = 1.0, h: float = 0.0,
                precision="fp64", tol: float | None = None, layers=None, **plan_kw) -> dict:
    """Sweep-optimise the isometries of one network (a site tensor T0, or the
    Ising model at (beta, J, h)).  Returns dict(lnz_hotrg, lnz (after each
    sweep), lnz_final, isometries (per step, w[x1, x2, a]), sweeps).

    ``layers``: the steps updated in each sweep, inner to outer (default all).
    ``tol``: stop before n_sweeps once a sweep changes ln Z/N by at most tol
    times the total change since the HOTRG start (the main text sweeps "until
    the results converge", with a convergence criterion of 1e-4 for the
    relative errors of Fig. 2; this reading measures it against the
    improvement itself, which needs no exact value)."""
    if (T0 is None) == (beta is None):
        raise ValueError("give exactly one of T0 or beta")

    def forward(p):
        if T0 is not None:
            return p.forward_tensor(np.asarray(T0, dtype=np.float64))[0]
        return p.forward_ising(beta, J, h)[0]

    with Plan(d0, d_cut, n_steps, precision, want_grad=True, **plan_kw) as p0:
        lnz_hotrg = forward(p0)
        ws = p0.isometries()
    history = []
    with Plan(d0, d_cut, n_steps, precision, want_grad=True, fixed_w_grad=True, w_given=True,
              **plan_kw) as p:
        p.set_isometries(ws)
        ks = list(layers) if layers is not None else list(range(1, n_steps + 1))
        for _ in range(n_sweeps):
            for k in ks:
                for _ in range(n_inner):
                    forward(p)
                    p.backward()
                    p.mera_update(k)
            history.append(forward(p))
            if tol is not None and len(history) >= 2:
                change = abs(history[-1] - history[-2])
                if change <= tol * abs(history[-1] - lnz_hotrg):
                    break
        ws = p.isometries()
    return dict(lnz_hotrg=lnz_hotrg, lnz=history,
                lnz_final=history[-1] if history else lnz_hotrg, isometries=ws,
                sweeps=len(history))


def lbfgs_sweeps(d0: int, d_cut: int, n_steps: int, n_sweeps: int, n_iter: int,
                 history: int = 10, T0=None, beta: float | None = None, J: float = 1.0,
                 h: float = 0.0, precision="fp64", layers=None, step0: float = 0.1,
                 c1: float = 1e-4, **plan_kw) -> dict:
    """Quasi-Newton alternative to the MERA update (SM Sec. D): starting from
    HOTRG, each layer in turn (inner to outer, ``layers`` default all) gets
    n_iter L-BFGS iterations on w_k = Q exp(B) E with the others fixed, for
    n_sweeps sweeps.  Returns dict(lnz_hotrg, lnz (after each sweep),
    layer_hist (ln Z/N per accepted iterate, per layer visit), evals,
    isometries)."""
    if (T0 is None) == (beta is None):
        raise ValueError("give exactly one of T0 or beta")

    def forward(p):
        if T0 is not None:
            return p.forward_tensor(np.asarray(T0, dtype=np.float64))[0]
        return p.forward_ising(beta, J, h)[0]

    with Plan(d0, d_cut, n_steps, precision, want_grad=True, **plan_kw) as p0:
        lnz_hotrg = forward(p0)
        ws = p0.isometries()
    history_lnz, layer_hist, evals = [], [], 0
    with Plan(d0, d_cut, n_steps, precision, want_grad=True, fixed_w_grad=True, w_given=True,
              **plan_kw) as p:
        p.set_isometries(ws)
        forward(p)
        ks = list(layers) if layers is not None else list(range(1, n_steps + 1))
        with LBFGS(p, history) as opt:
            for _ in range(n_sweeps):
                for k in ks:
                    f, ev = opt.layer(k, n_iter, step0=step0, c1=c1)
                    layer_hist.append(f)
                    evals += ev
                history_lnz.append(forward(p))
        ws = p.isometries()
    return dict(lnz_hotrg=lnz_hotrg, lnz=history_lnz, layer_hist=layer_hist, evals=evals,
                isometries=ws)
