"""Differentiable-TRG sweep optimisation of the HOTRG isometries, plain FP64
on the CPU (NumPy + LAPACK).

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the
product path.

The HOTRG network of ``oracle.hotrg`` is a function of the site tensor T0 and
of the isometries {w_k}.  HOTRG chooses each w_k locally (leading
eigenvectors of the Gram matrix of step k).  Differentiable TRG (main text,
"Differentiable tensor renormalization group"; Eq. (1)) treats the w_k as
parameters and improves them with the environment of each one:

    E_w^(k) = wbar_k / N_k,   wbar_k = d Z / d w_k,

obtained by one backward sweep with every w held fixed (``hotrg_backward``
with ``fixed_w=True``; it returns d(ln Z/N)/d w_k, a positive multiple of
dZ/dw_k, which has the same singular vectors).  The MERA update (main text,
after Eq. (1)) replaces w_k by the isometry that maximises Tr(E_w^T w) for
the current environment:

    E_w = U S V^T (thin SVD)   ->   w_k = U V^T,

whose value Tr(E_w^T U V^T) = sum of the singular values is the maximum over
all isometries of that shape (von Neumann's trace inequality).  Because Z is
not linear in w_k (w_k enters twice per step and every later tensor depends
on it), one MERA update is repeated n_inner times with a fresh environment,
and the layers are swept n_sweeps times.

Readings (the paper does not fix them):
* "inner to outer layers": the first coarse-graining step is the innermost
  function of the composition T_n(...T_1(T0)), so a sweep updates
  k = 1, 2, ..., n in that order;
* every forward inside the sweep uses the current isometries as given (no
  eigensolve), with the same Frobenius normalisation and trace as HOTRG, so
  ln Z / N of a sweep is directly comparable with the HOTRG one;
* the sweep starts from the HOTRG isometries.
"""
from __future__ import annotations

import math

import numpy as np

from . import hotrg


def forward_fixed_w(T0, ws):
    """HOTRG forward with every isometry given (ws[k-1] has shape
    (X, X, D') for step k).  Returns a dict in the format of
    ``hotrg.hotrg_forward(..., keep=True)`` (checkpoints without the
    eigenpairs), suitable for ``hotrg.hotrg_backward(fwd, fixed_w=True)``."""
    T = np.array(T0, dtype=np.float64)
    n = len(ws)
    S = 0.0
    log_norms, ckpt = [], []
    for k in range(1, n + 1):
        if k > 1:
            T = hotrg.orient(T)
        X = T.shape[0]
        w = np.asarray(ws[k - 1], dtype=np.float64)
        if w.shape[:2] != (X, X):
            raise ValueError(f"isometry of step {k} has shape {w.shape}, expected ({X}, {X}, D')")
        Tn = hotrg.hotrg_step(T, w)
        c = float(np.linalg.norm(Tn))
        log_norms.append(math.log(c))
        S += math.log(c) / 2.0 ** k
        ckpt.append(dict(T=T, w=w, c=c, Dp=w.shape[2]))
        T = Tn / c
    tr = hotrg.trace(T)
    lnz = S + math.log(abs(tr)) / 2.0 ** n
    return dict(lnz=lnz, log_norms=log_norms, trace=tr, trace_sign=1 if tr >= 0 else -1,
                ckpt=ckpt, T_final=T, n_steps=n)


def mera_update(E):
    """The isometry maximising Tr(E^T w) over all w with w^T w = I, for an
    environment E of shape (X, X, D'): the polar factor U V^T of E."""
    X1, X2, Dp = E.shape
    U, _, Vt = np.linalg.svd(E.reshape(X1 * X2, Dp), full_matrices=False)
    return (U @ Vt).reshape(X1, X2, Dp)


def environments(T0, ws):
    """ln Z / N and the environments d(ln Z/N)/d w_k of the network with
    the given isometries."""
    fwd = forward_fixed_w(T0, ws)
    _, wbars = hotrg.hotrg_backward(fwd, fixed_w=True, return_wbar=True)
    return fwd["lnz"], wbars


def dtrg_sweeps(T0, d_cut: int, n_steps: int, n_sweeps: int, n_inner: int = 1):
    """Start from HOTRG and run n_sweeps sweeps of MERA updates over the
    layers k = 1..n, each repeated n_inner times with a fresh environment.

    Returns dict(ws, lnz_hotrg, lnz (after each sweep), lnz_final)."""
    base = hotrg.hotrg_forward(T0, d_cut, n_steps, keep=True)
    ws = [ck["w"].copy() for ck in base["ckpt"]]
    history = []
    for _ in range(n_sweeps):
        for k in range(1, n_steps + 1):
            for _ in range(n_inner):
                _, wbars = environments(T0, ws)
                ws[k - 1] = mera_update(wbars[k - 1])
        history.append(forward_fixed_w(T0, ws)["lnz"])
    return dict(ws=ws, lnz_hotrg=base["lnz"], lnz=history,
                lnz_final=history[-1] if history else base["lnz"])
