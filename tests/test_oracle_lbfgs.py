"""Pins of the L-BFGS isometry optimiser (oracle/lbfgs.py): the exponential
parametrisation, its gradient against finite differences, the two-loop
recursion on quadratics, monotone ascent and the gain over HOTRG."""
import math

import numpy as np
import pytest

from oracle import dtrg, exact, hotrg, ising, lbfgs


def _w0(d_cut=6, n=6, beta=0.40):
    T0 = ising.ising_T0(beta, 1.0, 0.0)
    ws = [ck["w"] for ck in hotrg.hotrg_forward(T0, d_cut, n)["ckpt"]]
    return T0, ws


def test_completion_and_exponential_stay_isometric():
    _, ws = _w0()
    w = ws[3]
    X, _, Dp = w.shape
    Q = lbfgs.completion(w)
    N = X * X
    assert np.abs(Q.T @ Q - np.eye(N)).max() < 1e-13
    assert np.abs(Q[:, :Dp] - w.reshape(N, Dp)).max() < 1e-14
    rng = np.random.default_rng(0)
    b = rng.standard_normal(N * (N - 1) // 2)
    W = lbfgs.isometry(Q, b, X, Dp).reshape(N, Dp)
    assert np.abs(W.T @ W - np.eye(Dp)).max() < 1e-12
    assert np.abs(lbfgs.isometry(Q, 0 * b, X, Dp) - w).max() < 1e-14


def test_gradient_against_finite_differences():
    T0, ws = _w0()
    k = 4
    X, _, Dp = ws[k - 1].shape
    Q = lbfgs.completion(ws[k - 1])
    rng = np.random.default_rng(1)
    N = X * X
    b0 = 0.05 * rng.standard_normal(N * (N - 1) // 2)

    def f(b):
        w2 = list(ws)
        w2[k - 1] = lbfgs.isometry(Q, b, X, Dp)
        return dtrg.forward_fixed_w(T0, w2)["lnz"]

    w2 = list(ws)
    w2[k - 1] = lbfgs.isometry(Q, b0, X, Dp)
    _, wbars = dtrg.environments(T0, w2)
    g = lbfgs.gradient_b(Q, b0, wbars[k - 1])
    for i in rng.choice(b0.size, 10, replace=False):
        e = np.zeros_like(b0)
        e[i] = 1e-6
        fd = (f(b0 + e) - f(b0 - e)) / 2e-6
        assert abs(fd - g[i]) < 1e-9 + 1e-6 * np.abs(g).max()


@pytest.mark.parametrize("k", [5, 6])
def test_gradient_blocks_at_the_base_point(k):
    # at B = 0, rotations within the discarded block do not touch w; rotations
    # within the kept block of the last two layers are a gauge of the final
    # trace (for earlier layers the later, fixed isometries are not
    # co-rotated, so those are real changes of the network)
    T0, ws = _w0()
    X, _, Dp = ws[k - 1].shape
    N = X * X
    Q = lbfgs.completion(ws[k - 1])
    _, wbars = dtrg.environments(T0, ws)
    G = lbfgs.unpack(lbfgs.gradient_b(Q, np.zeros(N * (N - 1) // 2), wbars[k - 1]), N)
    assert np.abs(G[Dp:, Dp:]).max() == 0.0
    assert np.abs(G[:Dp, :Dp]).max() < 1e-12 * np.abs(G).max()
    assert np.abs(G[Dp:, :Dp]).max() > 0


def test_two_loop_maximises_a_concave_quadratic():
    rng = np.random.default_rng(2)
    n = 12
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    c = rng.standard_normal(n)
    fg = lambda x: (-0.5 * x @ A @ x + c @ x, -A @ x + c)
    x, hist, _ = lbfgs.maximise(fg, np.zeros(n), 60, m=12)
    assert np.abs(x - np.linalg.solve(A, c)).max() < 1e-9
    assert all(b >= a for a, b in zip(hist, hist[1:]))


def test_two_loop_reproduces_bfgs_inverse_on_stored_pairs():
    # with every pair stored, H y_newest = s_newest (the secant equation of the
    # newest pair holds exactly for the L-BFGS matrix)
    rng = np.random.default_rng(3)
    n = 8
    S = [rng.standard_normal(n) for _ in range(4)]
    A = np.diag(np.linspace(1, 5, n))
    Y = [A @ s for s in S]
    assert np.abs(lbfgs.two_loop(Y[-1], S, Y) - S[-1]).max() < 1e-12


def test_layer_sweeps_ascend_and_improve_hotrg_off_criticality():
    beta = 0.40
    T0 = ising.ising_T0(beta, 1.0, 0.0)
    r = lbfgs.lbfgs_sweeps(T0, 6, 16, n_sweeps=1, n_iter=5)
    for h in r["layer_hist"]:
        assert all(b >= a - 1e-15 for a, b in zip(h, h[1:]))
    ex = exact.onsager_lnz(beta)
    assert abs(r["lnz"][-1] - ex) < 0.5 * abs(r["lnz_hotrg"] - ex)
    for w in r["ws"]:
        X1, X2, Dp = w.shape
        m = w.reshape(X1 * X2, Dp)
        assert np.abs(m.T @ m - np.eye(Dp)).max() < 1e-12


def test_converged_layer_is_stationary_on_the_stiefel_manifold():
    # after enough iterations on one layer, the environment has no component
    # that a rotation of w could use: (1 - w w^T) E = 0 and w^T E symmetric
    T0, ws = _w0(d_cut=4, n=5)
    k = 3
    r = lbfgs.lbfgs_sweeps(T0, 4, 5, n_sweeps=1, n_iter=100, layers=[k])
    _, wbars = dtrg.environments(T0, r["ws"])
    w = r["ws"][k - 1]
    X1, X2, Dp = w.shape
    W = w.reshape(X1 * X2, Dp)
    E = wbars[k - 1].reshape(X1 * X2, Dp)
    scale = np.abs(E).max()
    assert np.abs(E - W @ (W.T @ E)).max() < 1e-8 * scale
    S = W.T @ E
    assert np.abs(S - S.T).max() < 1e-8 * scale
