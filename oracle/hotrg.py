"""Plain FP64 HOTRG forward and backward on the CPU (NumPy + LAPACK).

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the
product path.

Conventions
-----------
* A tensor is ``T[l, r, u, d]`` (row-major, d fastest).  Horizontal legs
  l, r have dimension X; vertical legs u, d have dimension Y.
* One coarse-graining step merges two tensors stacked vertically, exactly
  as the HOTRG step equation of SM Sec. B writes it: the upper tensor is
  T[x1, x1', y, j], the lower one T[x2, x2', j, y'], the shared vertical bond
  j is summed, and the new tensor is

      T'[alpha, beta, y, y'] = sum T[x1,x1',y,j] T[x2,x2',j,y']
                                   w[x1,x2,alpha] w[x1',x2',beta].

* Steps alternate direction (main text Fig. 1a, "w introduced along both
  directions"): before every step after the first the tensor is
  re-oriented ``T[l, r, u, d] -> T[u, d, l, r]``, so "vertical" always
  means the merge direction.  After n steps the last tensor stands for a
  periodic torus of 2^floor(n/2) (x) by 2^ceil(n/2) (y) sites.
* The isometry w comes from the local higher-order SVD (SM Sec. B, last
  sentence of the forward paragraph).  The HOSVD subspace of the merged
  pair M = T.T along (x1, x2) equals the leading eigenvectors of its Gram
  matrix G = M M^T, which is assembled from two half-environments:

      A[x1, j, x1'', j'] = sum_{x1', y}  T[x1,x1',y,j]  T[x1'',x1',y,j']
      B[x2, j, x2'', j'] = sum_{x2', y'} T[x2,x2',j,y'] T[x2'',x2',j',y']
      G[(x1 x2), (x1'' x2'')] = sum_{j, j'} A[x1,j,x1'',j'] B[x2,j,x2'',j'].

  Eigenvalues are sorted in descending order and the leading
  D' = min(X^2, D_cut) eigenvectors are kept: w[x1, x2, a] = U[(x1 x2), a].
  Gauge: each eigenvector is flipped so that its largest-magnitude
  component (first one on ties) is positive.  Z does not depend on this
  choice; it is fixed only so that intermediate tensors are reproducible.
* Normalisation (implied by Z staying finite over 2^n sites, main text):
  after step k the new tensor is divided by its Frobenius norm c_k and
  ln c_k / 2^k is accumulated.  With N = 2^n sites,

      ln Z / N = sum_k ln c_k / 2^k + ln |sum_{x,y} T_n[x, x, y, y]| / 2^n.

Backward (reverse mode)
-----------------------
The SM Sec. B second-renormalization recursion carries the environment of
the local tensor from scale i+1 down to scale i through the Jacobian of
the HOTRG step (SM Sec. E: environment = derivative of Z, Jacobian of the
step, chain rule; the environment is the average over the upper and lower
copy).  This module differentiates the computed ln Z / N as a function of
T0 and carries

    E_k = 2^k * d(ln Z / N) / d T~_k        (T~_k = normalised tensor),

so that E_{k-1} = (1/2) * (adjoint of step k applied to E_k / c_k) -- the
factor 1/2 is the paper's average over the two copies.  The norms c_k are
held constant in the backward; this is exact because ln Z / N equals
ln |tr T_n^{raw}| / 2^n of the unnormalised chain, which differs from the
normalised one only by those constants.

Two gradient modes:
* full (default): w depends on T through the eigensolve, and the adjoint of
  the truncated eigensolve and of the Gram assembly is included;
* fixed_w: w is held fixed (the paper's view of w as independent
  parameters, SM Sec. E), giving the pure second-renormalization
  environment.

Adjoint of the truncated eigensolve (the paper relies on automatic
differentiation here and prints no formula; this is the standard
first-order eigenvector perturbation restricted as follows): ln Z is
invariant under w -> w O for any orthogonal O on the kept block, so the
kept x kept terms cancel exactly and are set to zero; only kept k x
discarded j pairs contribute,

    Gbar = U_disc [F o (U_disc^T wbar)] U_kept^T,  symmetrised,
    F[j, k] = (lam_k - lam_j) / ((lam_k - lam_j)^2 + eta),
    eta = eta_rel * lam_1^2   (eta_rel = 1e-12 by default),

which is the exact expression when lam_k - lam_j >> sqrt(eta).
"""
from __future__ import annotations

import math

import numpy as np

ETA_REL_DEFAULT = 1e-12
W_RULE_TIE = 1e-12   # relative tie band of the w_rule = 1 comparison


def orient(T: np.ndarray) -> np.ndarray:
    """Re-orient ``T[l, r, u, d] -> T[u, d, l, r]`` (an involution)."""
    return np.ascontiguousarray(T.transpose(2, 3, 0, 1))


def gram_halves(T: np.ndarray):
    """Half-environments A[x1, j, x1'', j'] and B[x2, j, x2'', j']."""
    A = np.einsum("aiyj,ciyk->ajck", T, T, optimize=True)
    B = np.einsum("bkjz,dkmz->bjdm", T, T, optimize=True)
    return A, B


def gram(T: np.ndarray) -> np.ndarray:
    """Environment Gram matrix G[(x1 x2), (x1'' x2'')], shape (X^2, X^2)."""
    X = T.shape[0]
    A, B = gram_halves(T)
    G = np.einsum("ajck,bjdk->abcd", A, B, optimize=True)
    return G.reshape(X * X, X * X)


def eigh_desc(G: np.ndarray):
    """All eigenpairs of the symmetric G, eigenvalues descending, each
    eigenvector sign-fixed (largest-|.| component positive, first on ties)."""
    lam, U = np.linalg.eigh(G)
    lam = lam[::-1].copy()
    U = U[:, ::-1].copy()
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(U.shape[1])])
    sgn[sgn == 0] = 1.0
    return lam, U * sgn


def hotrg_step(T: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The HOTRG step equation (SM Sec. B) for one vertical merge.

    T: (X, X, Y, Y); w: (X, X, X').  Returns T'[alpha, beta, y, y'] of shape
    (X', X', Y, Y).  The five-index sum is evaluated pairwise, one value of
    the free leg y at a time (only to bound memory):
        U_y[x1', j, x2, alpha]   = sum_{x1} T[x1, x1', y, j] w[x1, x2, alpha]
        V_y[x1', alpha, x2', y'] = sum_{x2, j} U_y[x1', j, x2, alpha] T[x2, x2', j, y']
        T'[alpha, beta, y, y']   = sum_{x1', x2'} V_y[x1', alpha, x2', y'] w[x1', x2', beta]
    """
    X, _, Y, _ = T.shape
    Xp = w.shape[2]
    out = np.empty((Xp, Xp, Y, Y))
    for y in range(Y):
        Uy = np.tensordot(T[:, :, y, :], w, axes=([0], [0]))        # [i, j, b, A]
        Vy = np.tensordot(Uy, T, axes=([2, 1], [0, 2]))              # [i, A, k, z]
        out[:, :, y, :] = np.tensordot(Vy, w, axes=([0, 2], [0, 1])).transpose(0, 2, 1)
    return out


def swap_lr(T: np.ndarray) -> np.ndarray:
    """T[l, r, u, d] -> T[r, l, u, d] (an involution)."""
    return np.ascontiguousarray(T.transpose(1, 0, 2, 3))


def choose_isometry(T: np.ndarray, d_cut: int, w_rule: int = 0):
    """Eigenpairs of the Gram matrix that gives the isometry of this step and
    the side it came from (0 = left, 1 = right).

    w_rule 0: the left Gram matrix, always.  w_rule 1 (Xie2012's rule): the
    HOSVD of the merged pair along its left bond (x1 x2) and along its right
    bond (x1' x2'); the side whose discarded eigenvalues sum to less (the two
    Gram matrices have the same trace) gives w, the left one on a tie.  A tie
    is a difference of at most W_RULE_TIE times the trace: on a tensor whose
    two sides have the same spectrum the sums differ by rounding only.  The
    right Gram matrix is the left one of the tensor with l and r exchanged."""
    X = T.shape[0]
    lam, U = eigh_desc(gram(T))
    Dp = min(X * X, d_cut)
    if w_rule == 1 and Dp < X * X:
        lamR, UR = eigh_desc(gram(swap_lr(T)))
        eL, eR = float(np.sum(lam[Dp:])), float(np.sum(lamR[Dp:]))
        if eL - eR > W_RULE_TIE * float(np.sum(lam)):
            return lamR, UR, 1
    return lam, U, 0


def trace(T: np.ndarray) -> float:
    """Periodic self-contraction sum_{x, y} T[x, x, y, y] (main text: the
    single remaining tensor's self-contraction gives Z)."""
    return float(np.einsum("xxyy->", T))


def hotrg_forward(T0, d_cut: int, n_steps: int, keep: bool = True, w_override=None,
                  w_rule: int = 0):
    """HOTRG forward.  Returns a dict with

    lnz         ln Z / N (N = 2^n_steps sites)
    log_norms   [ln c_1, ..., ln c_n]
    trace       sum T~_n[x, x, y, y] of the last normalised tensor
    trace_sign  sign of that trace
    trunc_err   per step, sum of discarded eigenvalues / sum of all
    cut_gap     per step, (lam_D' - lam_D'+1) / lam_1 (inf if nothing cut)
    ckpt        (keep=True) per step dict(T, w, lam, U, c, Dp): T is the
                oriented input of the step, U all sign-fixed eigenvectors
    T_final     the last normalised tensor

    ``w_override(k, X, Dp, lam, U) -> w`` may replace the isometry of step k
    (used only by invariance pins).  ``w_rule``: which Gram matrix gives the
    isometry (see ``choose_isometry``); the checkpoint records the side.
    """
    T = np.array(T0, dtype=np.float64)
    if T.ndim != 4 or T.shape[0] != T.shape[1] or T.shape[2] != T.shape[3]:
        raise ValueError("T0 must have shape (X, X, Y, Y)")
    S = 0.0
    log_norms, trunc, gaps, ckpt = [], [], [], []
    for k in range(1, n_steps + 1):
        if k > 1:
            T = orient(T)
        X = T.shape[0]
        N = X * X
        lam, U, side = choose_isometry(T, d_cut, w_rule)
        Dp = min(N, d_cut)
        if w_override is not None:
            w = w_override(k, X, Dp, lam, U)
        else:
            w = U[:, :Dp].reshape(X, X, Dp)
        Tn = hotrg_step(T, w)
        c = float(np.linalg.norm(Tn))
        log_norms.append(math.log(c))
        S += math.log(c) / 2.0 ** k
        total = float(np.sum(lam))
        trunc.append(float(np.sum(lam[Dp:])) / total if total != 0 else 0.0)
        gaps.append(float((lam[Dp - 1] - lam[Dp]) / lam[0]) if Dp < N else math.inf)
        if keep:
            ckpt.append(dict(T=T, w=w, lam=lam, U=U, c=c, Dp=Dp, side=side))
        T = Tn / c
    tr = trace(T)
    lnz = S + math.log(abs(tr)) / 2.0 ** n_steps
    return dict(lnz=lnz, log_norms=log_norms, trace=tr, trace_sign=1 if tr >= 0 else -1,
                trunc_err=trunc, cut_gap=gaps, ckpt=ckpt, T_final=T, n_steps=n_steps,
                d_cut=d_cut)


def hotrg_step_backward(T, w, Tbar_out):
    """Adjoint of ``hotrg_step`` (SM Sec. E, Jacobian of the step).

    Tbar_out = d L / d T'.  Returns (Tbar, wbar): the sum of the upper- and
    lower-copy contributions to d L / d T (T enters twice), and d L / d w
    (w enters twice: w_L carries alpha, w_R carries beta).  Evaluated one
    value of y at a time like the forward.
    """
    X, _, Y, _ = T.shape
    Tbar = np.zeros_like(T)
    wbar = np.zeros_like(w)
    for y in range(Y):
        Tby = Tbar_out[:, :, y, :]                                   # [A, B, z]
        Ty = T[:, :, y, :]                                           # [a, i, j]
        Ry = np.tensordot(Ty, w, axes=([0], [0]))                    # [i, j, b, A]
        Vy = np.tensordot(Ry, T, axes=([2, 1], [0, 2]))              # [i, A, k, z]
        Py = np.tensordot(Tby, w, axes=([1], [2]))                   # [A, z, i, k]
        Qy = np.tensordot(Py, T, axes=([3, 1], [1, 3]))              # [A, i, b, j]
        # upper copy: Tbar_u[a, i, y, j] = sum_{A, b} w[a, b, A] Q_y[A, i, b, j]
        Tbar[:, :, y, :] += np.tensordot(w, Qy, axes=([1, 2], [2, 0]))
        # lower copy: Tbar_d[b, k, j, z] += sum_{i, A} R_y[i, j, b, A] P_y[A, z, i, k]
        Tbar += np.tensordot(Ry, Py, axes=([0, 3], [2, 0])).transpose(1, 3, 0, 2)
        # w carrying alpha: sum_{i, j} T[a, i, y, j] Q_y[A, i, b, j]
        wbar += np.tensordot(Ty, Qy, axes=([1, 2], [1, 3])).transpose(0, 2, 1)
        # w carrying beta: sum_{A, z} V_y[i, A, k, z] Tbar'[A, B, y, z]
        wbar += np.tensordot(Vy, Tby, axes=([1, 3], [0, 2]))
    return Tbar, wbar


def eigh_backward(lam, U, Dp, wbar, eta_rel=ETA_REL_DEFAULT):
    """Adjoint of w = U[:, :Dp] through the symmetric eigensolve (kept x
    discarded pairs only, broadened; see the module docstring).  Returns the
    symmetric Gbar (N x N)."""
    N = U.shape[0]
    Wb = wbar.reshape(N, Dp)
    if Dp >= N:
        return np.zeros((N, N))
    Uk, Ud = U[:, :Dp], U[:, Dp:]
    diff = lam[None, :Dp] - lam[Dp:, None]             # lam_k - lam_j, [j, k]
    eta = eta_rel * lam[0] ** 2
    F = diff / (diff * diff + eta)
    Gb = Ud @ (F * (Ud.T @ Wb)) @ Uk.T
    return 0.5 * (Gb + Gb.T)


def gram_backward(T, Gbar):
    """Adjoint of ``gram``: d L / d T from d L / d G (through A and B)."""
    X = T.shape[0]
    A, B = gram_halves(T)
    Gb4 = Gbar.reshape(X, X, X, X)                     # [x1, x2, x1'', x2'']
    Abar = np.einsum("abcd,bjdk->ajck", Gb4, B, optimize=True)
    Bbar = np.einsum("abcd,ajck->bjdk", Gb4, A, optimize=True)
    Tbar = np.einsum("ajck,ciyk->aiyj", Abar, T, optimize=True)
    Tbar += np.einsum("ckaj,ciyk->aiyj", Abar, T, optimize=True)
    Tbar += np.einsum("bjdm,dkmz->bkjz", Bbar, T, optimize=True)
    Tbar += np.einsum("dmbj,dkmz->bkjz", Bbar, T, optimize=True)
    return Tbar


def hotrg_backward(fwd, fixed_w: bool = False, eta_rel: float = ETA_REL_DEFAULT,
                   return_wbar: bool = False):
    """d(ln Z / N) / d T0 from a ``hotrg_forward(..., keep=True)`` result.

    With ``return_wbar`` also returns the list of d(ln Z/N)/d w_k (per step,
    the total over the two places w_k enters), i.e. the adjoint of main-text
    Eq. (1) divided by N.
    """
    n = fwd["n_steps"]
    Tn = fwd["T_final"]
    X, _, Y, _ = Tn.shape
    E = np.zeros_like(Tn)                     # E_n = 2^n dL/dT~_n
    for x in range(X):
        for y in range(Y):
            E[x, x, y, y] = 1.0 / fwd["trace"]
    wbars = [None] * n
    for k in range(n, 0, -1):
        ck = fwd["ckpt"][k - 1]
        T, w, c = ck["T"], ck["w"], ck["c"]
        Tbar, wbar = hotrg_step_backward(T, w, E / c)   # 2^k dL/dT, 2^k dL/dw
        wbars[k - 1] = wbar / 2.0 ** k
        if not fixed_w:
            Gbar = eigh_backward(ck["lam"], ck["U"], ck["Dp"], wbar, eta_rel)
            if np.any(Gbar):
                if ck.get("side", 0) == 1:
                    Tbar = Tbar + swap_lr(gram_backward(swap_lr(T), Gbar))
                else:
                    Tbar = Tbar + gram_backward(T, Gbar)
        E = 0.5 * (orient(Tbar) if k > 1 else Tbar)
    if return_wbar:
        return E, wbars
    return E
