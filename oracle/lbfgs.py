"""Quasi-Newton (L-BFGS) optimisation of the HOTRG isometries with the
isometric constraint built into an exponential parametrisation, plain FP64
on the CPU (NumPy / SciPy).

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the
product path.

SM Sec. D: the isometry of layer k is written through an antisymmetric
N x N matrix B (N = X^2), w = exp(B) truncated to its first D' columns, and
the standard gradient-based L-BFGS method updates B to maximise Z, given
the gradient E_w = wbar / N_k of main-text Eq. (1).

Readings (the paper fixes none of them):
* Base point.  w_k(B) = Q_k exp(B) E, E = the first D' columns of the N x N
  identity, Q_k an orthogonal N x N matrix whose first D' columns are the
  current w_k (the complete QR factor of w_k, columns sign-fixed so that
  Q_k E = w_k).  B = 0 is then the current isometry; the paper's exp(B) is
  the case Q_k = I.  Which completion Q_k takes does not matter: another one
  is Q_k P with P orthogonal and P E = E, and B -> P^T B P is an orthogonal
  change of the L-BFGS variables, which leaves the iteration unchanged.
* Variables: the strictly lower triangle b of B (B = b - b^T), Euclidean
  inner product.  The gradient of f(B) = ln Z / N is
      d f / d b_ij = G_ij - G_ji,   G = L_exp(B^T, Q_k^T wbar_k E^T),
  L_exp(A, C) the Frechet derivative of the matrix exponential at A in the
  direction C (the adjoint of L_exp(B, .) is L_exp(B^T, .)), wbar_k =
  d(ln Z/N)/d w_k of the backward with every isometry held fixed.
* L-BFGS: the two-loop recursion (Nocedal and Wright, Numerical
  Optimization, 2nd ed., Algorithm 7.4) on -f with m stored pairs and
  H_0 = (s^T y / y^T y) I; the first iteration (no pair yet) scales the
  steepest-ascent direction to step0 / ||g|| (a rotation of step0
  radians).  Backtracking line search from the full step, halving until
  the Armijo condition f(b + a p) >= f(b) + c1 a g^T p holds (at most
  max_backtracks halvings, else the iteration ends the run).  A pair with
  s^T y >= 0 (no negative curvature of -f) is not stored.
* Layers: like the MERA sweeps, one layer at a time with the others held
  fixed, inner to outer, n_iter iterations per layer per sweep; after a
  layer's iterations its base point moves to the new isometry
  (Q_k <- Q_k exp(B), B <- 0) and its history is dropped.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm, expm_frechet

from . import dtrg, hotrg


def completion(w: np.ndarray) -> np.ndarray:
    """Orthogonal N x N matrix Q with Q[:, :D'] = w (w: X x X x D' with
    orthonormal columns over (x1 x2))."""
    X1, X2, Dp = w.shape
    W = w.reshape(X1 * X2, Dp)
    Q, R = np.linalg.qr(W, mode="complete")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    Q[:, :Dp] *= sgn
    return Q


def unpack(b: np.ndarray, N: int) -> np.ndarray:
    B = np.zeros((N, N))
    B[np.tril_indices(N, -1)] = b
    return B - B.T


def isometry(Q: np.ndarray, b: np.ndarray, X: int, Dp: int) -> np.ndarray:
    N = X * X
    return (Q @ expm(unpack(b, N))[:, :Dp]).reshape(X, X, Dp)


def gradient_b(Q: np.ndarray, b: np.ndarray, wbar: np.ndarray) -> np.ndarray:
    """d f / d b from wbar = d f / d w (X x X x D')."""
    N = Q.shape[0]
    Dp = wbar.shape[2]
    C = np.zeros((N, N))
    C[:, :Dp] = Q.T @ wbar.reshape(N, Dp)
    B = unpack(b, N)
    _, G = expm_frechet(B.T, C)
    il = np.tril_indices(N, -1)
    return G[il] - G.T[il]


def two_loop(g: np.ndarray, S, Y) -> np.ndarray:
    """H g for the L-BFGS inverse-Hessian approximation of the stored pairs
    (s_i, y_i) (oldest first), H_0 = (s^T y / y^T y) I of the newest pair."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        alphas.append(a)
        q -= a * y
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    r = gamma * q
    for (s, y), a in zip(zip(S, Y), reversed(alphas)):
        rho = 1.0 / float(y @ s)
        beta = rho * float(y @ r)
        r += (a - beta) * s
    return r


def maximise(fg, x0: np.ndarray, n_iter: int, m: int = 10, c1: float = 1e-4,
             step0: float = 0.1, max_backtracks: int = 30):
    """L-BFGS ascent of f from x0; fg(x) -> (f, g).  Returns (x, [f per
    accepted iterate, starting with f(x0)], evaluations)."""
    x = np.array(x0, dtype=np.float64)
    f, g = fg(x)
    hist = [f]
    S, Y = [], []
    evals = 1
    for _ in range(n_iter):
        gn = float(np.linalg.norm(g))
        if gn == 0.0:
            break
        # ascent direction p = H g (H approximates the inverse Hessian of -f, so
        # the descent direction of -f, -H(-g), is H g)
        p = two_loop(g, S, Y) if S else (step0 / gn) * g
        slope = float(g @ p)
        if slope <= 0.0:                  # not an ascent direction: restart
            S, Y = [], []
            p = (step0 / gn) * g
            slope = float(g @ p)
        a = 1.0
        ok = False
        for _ in range(max_backtracks + 1):
            xn = x + a * p
            fn, gn_vec = fg(xn)
            evals += 1
            if fn >= f + c1 * a * slope:
                ok = True
                break
            a *= 0.5
        if not ok:
            break
        s = xn - x
        y = g - gn_vec                    # gradient change of -f
        if float(s @ y) > 0.0:
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn_vec
        hist.append(f)
    return x, hist, evals


def lbfgs_sweeps(T0, d_cut: int, n_steps: int, n_sweeps: int, n_iter: int, m: int = 10,
                 step0: float = 0.1, c1: float = 1e-4, layers=None):
    """Start from HOTRG and optimise the isometries layer by layer with
    L-BFGS in the exponential parametrisation.  Returns dict(ws, lnz_hotrg,
    lnz (after each sweep), layer_hist (per layer visit, f per iterate))."""
    base = hotrg.hotrg_forward(T0, d_cut, n_steps, keep=True)
    ws = [ck["w"].copy() for ck in base["ckpt"]]
    ks = list(layers) if layers is not None else list(range(1, n_steps + 1))
    history, layer_hist = [], []
    for _ in range(n_sweeps):
        for k in ks:
            X, _, Dp = ws[k - 1].shape
            Q = completion(ws[k - 1])

            def fg(b, k=k, Q=Q, X=X, Dp=Dp):
                w2 = list(ws)
                w2[k - 1] = isometry(Q, b, X, Dp)
                lnz, wbars = dtrg.environments(T0, w2)
                return lnz, gradient_b(Q, b, wbars[k - 1])

            P = X * X * (X * X - 1) // 2
            b, hist, _ = maximise(fg, np.zeros(P), n_iter, m=m, c1=c1, step0=step0)
            ws[k - 1] = isometry(Q, b, X, Dp)
            layer_hist.append(hist)
        history.append(dtrg.forward_fixed_w(T0, ws)["lnz"])
    return dict(ws=ws, lnz_hotrg=base["lnz"], lnz=history, layer_hist=layer_hist)
