"""Scheme (b) of differentiable TRG: vertical-only renormalisation of a
translation-invariant MPO (exponential cooling of a density matrix), plain
FP64 on the CPU (NumPy + LAPACK).

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the
product path.

Main text Fig. 1b: only the vertical direction is renormalised, which leaves
a one-dimensional structure that is contracted exactly.  For the density
matrix of a quantum chain (SM Sec. F) one vertical merge is the MPO product
rho(2 tau) = rho(tau) rho(tau): the HOTRG step equation of SM Sec. B with
the upper tensor's column index d summed against the lower tensor's row
index u, the doubled horizontal bonds compressed by the isometry w.  The
physical legs keep their dimension; only the horizontal bond grows, to
D' = min(X^2, D_cut).  No step re-orients the tensor.

Per step k (the merge and isometry of ``hotrg.hotrg_step`` /
``hotrg.gram`` / ``hotrg.eigh_desc``, the same local-HOSVD isometry of the
merged pair along its left bond), the new tensor is Frobenius-normalised,
T~_k = T'_k / c_k.  The free energy of the depth-k network is evaluated at
beta = 2^(k+1) tau as Tr[rho(2^k tau) rho(2^k tau)], the product of the two
copies contracted exactly (the one-dimensional structure of Fig. 1b; the
usual evaluation of exponential cooling, which needs no further truncation):

    out_k = sum_{j <= k} ln c_j / 2^j + ln lambda_max(A_k) / 2^(k+1),
    A_k[(x1 x2), (x1' x2')] = sum_{y, j} T~_k[x1, x1', y, j] T~_k[x2, x2', j, y],

where lambda_max is the dominant eigenvalue of the cell transfer matrix of
the exact product (Tr_phys over a ring of L cells is Tr A^L, and
(1/L) ln Tr A^L -> ln lambda_max).  out_k is ln Z per copy of T0 in the
2^(k+1)-deep network: ln Tr rho(2^(k+1) tau) per cell is 2^(k+1) out_k.
A_k is the transfer matrix of ``hotrg_step(T~_k, identity)``, the merge
with no truncation.

Backward: the same reverse-mode recursion as ``hotrg.hotrg_backward``
(E_k = 2^k d out / d T~_k, E_{k-1} = (1/2) adjoint of step k applied to
E_k / c_k, norms held constant, exact for the same reason), without the
re-orientation.  Its seed is one more step of that recursion through the
untruncated final product: with d ln lambda_max / d A = l r^T / (lambda l^T r)
(A r = lambda r, l^T A = lambda l^T),

    E_n = (1/2) adjoint of hotrg_step(., identity) at T~_n applied to
          delta_{y y'} l_a r_b / (lambda l^T r).

Differentiable TRG in scheme (b) (main text, XY-chain paragraph): while
cooling, after step k the isometries of the last n_d layers are optimised
by MERA updates (``dtrg.mera_update``) with the environments of out_k, the
free energy at the next temperature; n_d = 1 optimises the current layer
only.  Readings: the isometry of a new layer starts from the local HOSVD of
the (already optimised) network below it; a sweep visits the layers inner
to outer, n_inner updates each, n_sweeps sweeps per layer k.  (Optimising
against ln lambda_max of the single truncated tensor instead would give the
outermost isometry an environment of rank at most two, whose polar factor
the SVD leaves undetermined.)
"""
from __future__ import annotations

import math

import numpy as np

from . import dtrg, hotrg


def transfer_matrix(T: np.ndarray) -> np.ndarray:
    """M[x, x'] = sum_y T[x, x', y, y]."""
    return np.einsum("abyy->ab", T)


def identity_isometry(X: int) -> np.ndarray:
    """w[x1, x2, (x1 x2)] = 1: the merge that truncates nothing."""
    return np.eye(X * X).reshape(X, X, X * X)


def square_transfer(T: np.ndarray) -> np.ndarray:
    """A[(x1 x2), (x1' x2')] = sum_{y, j} T[x1, x1', y, j] T[x2, x2', j, y]:
    the cell transfer matrix of the exact product of two copies of T."""
    return transfer_matrix(hotrg.hotrg_step(T, identity_isometry(T.shape[0])))


def dominant(M: np.ndarray):
    """(lambda, l, r) of the eigenvalue of largest modulus of M with its left
    and right eigenvectors; the eigenvalue must be real and positive (the
    transfer matrix of a positive operator's trace)."""
    lam, R = np.linalg.eig(M)
    i = int(np.argmax(np.abs(lam)))
    lamL, Lv = np.linalg.eig(M.T)
    j = int(np.argmin(np.abs(lamL - lam[i])))
    val = lam[i]
    if abs(val.imag) > 1e-10 * abs(val) or val.real <= 0:
        raise ValueError(f"dominant eigenvalue {val} of the transfer matrix is not real positive")
    r = np.real(R[:, i])
    l = np.real(Lv[:, j])
    return float(val.real), l, r


def xtrg_forward(T0, d_cut: int, n_steps: int, ws=None, keep: bool = True,
                 evaluate: bool = True, w_rule: int = 0):
    """Vertical-only coarse-graining of the MPO cell tensor T0[l, r, u, d].

    ``ws``: isometries per step (w[x1, x2, a]); an entry None (or a list
    shorter than n_steps) means: take it from the local HOSVD of that step.
    Returns dict(lnz = out_n, lnz_steps = [out_1..out_n], log_norms, ckpt
    (per step dict(T, w, lam, U, c, Dp)), T_final, n_steps); with
    evaluate=False out_k is not formed (lnz None; for pins on finite rings
    of untruncated networks, whose exact product would be too large)."""
    T = np.array(T0, dtype=np.float64)
    if T.ndim != 4 or T.shape[0] != T.shape[1] or T.shape[2] != T.shape[3]:
        raise ValueError("T0 must have shape (X, X, Y, Y)")
    S = 0.0
    log_norms, lnz_steps, ckpt = [], [], []
    for k in range(1, n_steps + 1):
        X = T.shape[0]
        N = X * X
        w = ws[k - 1] if (ws is not None and k - 1 < len(ws)) else None
        lam = U = None
        side = 0
        if w is None:
            lam, U, side = hotrg.choose_isometry(T, d_cut, w_rule)
            Dp = min(N, d_cut)
            w = U[:, :Dp].reshape(X, X, Dp)
        w = np.asarray(w, dtype=np.float64)
        if w.shape[:2] != (X, X):
            raise ValueError(f"isometry of step {k} has shape {w.shape}, expected ({X}, {X}, D')")
        Tn = hotrg.hotrg_step(T, w)
        c = float(np.linalg.norm(Tn))
        log_norms.append(math.log(c))
        S += math.log(c) / 2.0 ** k
        if keep:
            ckpt.append(dict(T=T, w=w, lam=lam, U=U, c=c, Dp=w.shape[2], side=side))
        T = Tn / c
        if evaluate:
            lnz_steps.append(S + math.log(dominant(square_transfer(T))[0]) / 2.0 ** (k + 1))
    return dict(lnz=lnz_steps[-1] if evaluate else None, lnz_steps=lnz_steps, log_norms=log_norms, ckpt=ckpt,
                T_final=T, n_steps=n_steps)


def xtrg_backward(fwd, fixed_w: bool = False, eta_rel: float = hotrg.ETA_REL_DEFAULT,
                  return_wbar: bool = False):
    """d out_n / d T0 (and, with return_wbar, d out_n / d w_k per step) from
    an ``xtrg_forward(..., keep=True)`` result.  The full gradient (default)
    includes the adjoint of each step's eigensolve and Gram matrix; steps
    whose isometry was given count as fixed."""
    n = fwd["n_steps"]
    Tn = fwd["T_final"]
    X, _, Y, _ = Tn.shape
    lam, l, r = dominant(square_transfer(Tn))
    P = np.outer(l, r) / (lam * float(l @ r))    # d ln lambda / d A
    seed = np.einsum("ab,yz->abyz", P, np.eye(Y))
    Tbar, _ = hotrg.hotrg_step_backward(Tn, identity_isometry(X), seed)
    E = 0.5 * Tbar                               # E_n = 2^n d out / d T~_n
    wbars = [None] * n
    for k in range(n, 0, -1):
        ck = fwd["ckpt"][k - 1]
        T, w, c = ck["T"], ck["w"], ck["c"]
        Tbar, wbar = hotrg.hotrg_step_backward(T, w, E / c)
        wbars[k - 1] = wbar / 2.0 ** k
        if not fixed_w and ck["U"] is not None:
            Gbar = hotrg.eigh_backward(ck["lam"], ck["U"], ck["Dp"], wbar, eta_rel)
            if np.any(Gbar):
                if ck["side"] == 1:
                    Tbar = Tbar + hotrg.swap_lr(hotrg.gram_backward(hotrg.swap_lr(T), Gbar))
                else:
                    Tbar = Tbar + hotrg.gram_backward(T, Gbar)
        E = 0.5 * Tbar
    if return_wbar:
        return E, wbars
    return E


def ring_lnz(fwd, L: int) -> float:
    """ln Tr rho(2^n tau) on a ring of L cells from the normalised chain:
    L 2^n sum_j ln c_j / 2^j + ln Tr M~_n^L (pins on rings; for L a power of
    two above 64 the power is formed by normalised repeated squaring)."""
    n = fwd["n_steps"]
    S = sum(lc / 2.0 ** (j + 1) for j, lc in enumerate(fwd["log_norms"]))
    M = transfer_matrix(fwd["T_final"])
    if L > 64 and L & (L - 1) == 0:
        c = float(np.linalg.norm(M))
        P, acc = M / c, math.log(c)
        for _ in range(L.bit_length() - 1):
            P = P @ P
            c = float(np.linalg.norm(P))
            P /= c
            acc = 2.0 * acc + math.log(c)
        return L * 2.0 ** n * S + acc + math.log(float(np.trace(P)))
    return L * 2.0 ** n * S + math.log(float(np.trace(np.linalg.matrix_power(M, L))))


def environments(T0, ws):
    """out_n and d out_n / d w_k of the network with every isometry given."""
    fwd = xtrg_forward(T0, 0, len(ws), ws=ws)
    _, wbars = xtrg_backward(fwd, fixed_w=True, return_wbar=True)
    return fwd["lnz"], wbars


def dtrg_cooling(T0, d_cut: int, n_steps: int, n_d: int = 1, n_sweeps: int = 1,
                 n_inner: int = 1):
    """Exponential cooling with differentiable-TRG optimisation of the last
    n_d layers after every step (see the module docstring).

    Returns dict(lnz_steps = out_k after the optimisation at layer k,
    lnz_hotrg_steps = out_k of plain scheme (b), ws)."""
    base = xtrg_forward(T0, d_cut, n_steps)
    ws = []
    out = []
    for k in range(1, n_steps + 1):
        fwd = xtrg_forward(T0, d_cut, k, ws=ws)          # the new layer from its local HOSVD
        ws = [ck["w"].copy() for ck in fwd["ckpt"]]
        for _ in range(n_sweeps):
            for layer in range(max(1, k - n_d + 1), k + 1):
                for _ in range(n_inner):
                    _, wbars = environments(T0, ws)
                    ws[layer - 1] = dtrg.mera_update(wbars[layer - 1])
        out.append(xtrg_forward(T0, d_cut, k, ws=ws)["lnz"])
    return dict(lnz_steps=out, lnz_hotrg_steps=base["lnz_steps"], ws=ws)


def lnz_per_site(out_k: float, k: int, sites_per_cell: int = 2) -> float:
    """ln Z per physical site at beta = 2^k tau from out_k (ln Z per T0
    copy): ln Tr rho(2^k tau) per cell is 2^k out_k."""
    return 2.0 ** k * out_k / sites_per_cell
