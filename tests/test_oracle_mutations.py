"""The oracle's pins have teeth: each test plants a plausible mistake in the
oracle (on the CPU, via monkeypatch) and checks that an independent pin
detects it.  Only the oracle is mutated; the CUDA path is not involved."""
import math

import numpy as np
import pytest

from oracle import exact, hotrg, ising
import synth


def _anisotropic_T0():
    T0 = synth.random_symmetric_T0(1, 4)
    return T0 + 0.3 * np.einsum("l,r,u,d->lrud", np.arange(4.0) - 1.0, np.arange(4.0) - 1.0,
                                np.ones(4), np.ones(4))


def _torus_pin(T0, n):
    Lx, Ly = 2 ** (n // 2), 2 ** ((n + 1) // 2)
    return abs(hotrg.hotrg_forward(T0, 10 ** 6, n, keep=False)["lnz"]
               - exact.torus_lnz(T0, Lx, Ly) / (Lx * Ly))


def test_missing_reorientation_is_caught(monkeypatch):
    # two steps: with the re-orientation the network is the 2 x 2 torus; without
    # it both merges are vertical (a 1 x 4 torus), which the pin must tell apart
    T0 = _anisotropic_T0()
    assert _torus_pin(T0, 2) < 1e-12
    monkeypatch.setattr(hotrg, "orient", lambda T: np.ascontiguousarray(T))
    assert _torus_pin(T0, 2) > 1e-6


def test_site_tensor_field_without_beta_is_caught():
    # a plausible slip in SM Sec. A's weights: exp(h s) instead of exp(beta h s)
    b, h = 0.4, 0.2
    lnz_bf = exact.bruteforce(4, 4, b, 1.0, h)[0]
    assert abs(exact.torus_lnz(ising.ising_T0(b, 1.0, h), 4, 4) / 16 - lnz_bf) < 1e-13
    bad = ising.ising_T0(b, 1.0, h / b)          # = the tensor with exp(h s)
    assert abs(exact.torus_lnz(bad, 4, 4) / 16 - lnz_bf) > 1e-3


def _fd_check(T0, d_cut, n, entries):
    f = hotrg.hotrg_forward(T0, d_cut, n)
    g = hotrg.hotrg_backward(f)
    e = 1e-6
    worst = 0.0
    for idx in entries:
        tp, tm = T0.copy(), T0.copy()
        tp[idx] += e
        tm[idx] -= e
        fd = (hotrg.hotrg_forward(tp, d_cut, n, keep=False)["lnz"]
              - hotrg.hotrg_forward(tm, d_cut, n, keep=False)["lnz"]) / (2 * e)
        worst = max(worst, abs(g[idx] - fd))
    return worst / np.max(np.abs(g))


ENTRIES = [(0, 0, 0, 0), (1, 2, 0, 1), (2, 2, 1, 0), (0, 1, 2, 2), (1, 1, 1, 1)]


def test_dropped_eigensolve_adjoint_is_caught(monkeypatch):
    T0 = synth.random_symmetric_T0(0, 3)
    assert _fd_check(T0, 6, 6, ENTRIES) < 1e-6
    monkeypatch.setattr(hotrg, "eigh_backward", lambda lam, U, Dp, wbar, eta_rel=0: np.zeros((U.shape[0],) * 2))
    assert _fd_check(T0, 6, 6, ENTRIES) > 1e-4


def test_half_gram_adjoint_is_caught(monkeypatch):
    T0 = synth.random_symmetric_T0(0, 3)

    def half(T, Gbar):
        X = T.shape[0]
        A, B = hotrg.gram_halves(T)
        Gb4 = Gbar.reshape(X, X, X, X)
        Abar = np.einsum("abcd,bjdk->ajck", Gb4, B, optimize=True)
        return np.einsum("ajck,ciyk->aiyj", Abar, T, optimize=True)   # B-side terms dropped

    monkeypatch.setattr(hotrg, "gram_backward", half)
    assert _fd_check(T0, 6, 6, ENTRIES) > 1e-4


def test_missing_copy_average_is_caught(monkeypatch):
    # forgetting the 1/2 average over the two copies breaks the Euler identity
    T0 = synth.random_symmetric_T0(0, 3)
    f = hotrg.hotrg_forward(T0, 6, 6)
    assert abs(np.sum(T0 * hotrg.hotrg_backward(f)) - 1.0) < 1e-12
    # plant: every step's adjoint doubled, i.e. the 1/2 average dropped
    real_step = hotrg.hotrg_step_backward

    def no_average(T, w, Tbar_out):
        Tb, wb = real_step(T, w, Tbar_out)
        return 2.0 * Tb, 2.0 * wb

    monkeypatch.setattr(hotrg, "hotrg_step_backward", no_average)
    g_bad = hotrg.hotrg_backward(f)
    assert abs(np.sum(T0 * g_bad) - 1.0) > 0.5


def test_wrong_normalisation_weight_is_caught(monkeypatch):
    # accumulating ln c_k / 2^(k+1) instead of / 2^k breaks the exact small torus
    T0 = ising.ising_T0(0.41, 1.0, 0.03)
    assert _torus_pin(T0, 4) < 1e-13
    real = hotrg.hotrg_step

    def scaled(T, w):
        return 3.0 * real(T, w)      # a step that is off by a constant factor

    monkeypatch.setattr(hotrg, "hotrg_step", scaled)
    assert _torus_pin(T0, 4) > 1e-3
