"""Pins of the XY-chain oracle (oracle/xy.py) and of the scheme-(b)
vertical-only contraction (oracle/xtrg.py) against exact diagonalisation,
closed forms, dense Trotter products, finite differences and invariants."""
import math
import warnings

import numpy as np
import pytest

from oracle import dtrg, hotrg, xtrg, xy

warnings.filterwarnings("ignore", message=".*roundoff error.*")


@pytest.mark.parametrize("N", [4, 6, 8, 10])
@pytest.mark.parametrize("beta", [0.3, 1.0, 3.0])
def test_jordan_wigner_sectors_equal_exact_diagonalisation(N, beta):
    # SM Sec. G: the parity-projected free-fermion sectors; ED of the 2^N spin
    # Hamiltonian decides the sector momenta (see oracle/xy.py)
    assert abs(xy.lnz_exact_finite(N, beta) - xy.lnz_ed(N, beta)) < 1e-12


def test_other_sector_assignment_disagrees_with_ed():
    # periodic momenta in the even sector (the other reading) is off by O(1)
    N, beta = 6, 2.0
    n = np.arange(N)
    qp = 2 * math.pi * n / N
    qa = 2 * math.pi * (n + 0.5) / N
    ep, ea = np.cos(qp), np.cos(qa)
    z = (0.5 * (np.prod(1 + np.exp(-beta * ep)) + np.prod(1 - np.exp(-beta * ep))) +
         0.5 * (np.prod(1 + np.exp(-beta * ea)) - np.prod(1 - np.exp(-beta * ea))))
    assert abs(math.log(z) - xy.lnz_ed(N, beta)) > 1e-3


def test_infinite_chain_limits():
    # beta = 0: ln 2; high-temperature series ln 2 + beta^2 <cos^2 q> / 8 = ln 2 + beta^2 / 16
    assert abs(xy.lnz_exact_infinite(0.0) - math.log(2.0)) < 1e-15
    b = 0.01
    assert abs(xy.lnz_exact_infinite(b) - (math.log(2.0) + b * b / 16)) < 1e-10
    # the finite rings converge to the integral (exponentially fast at beta = 1)
    assert abs(xy.lnz_exact_finite(400, 1.0) / 400 - xy.lnz_exact_infinite(1.0)) < 1e-12
    # f(-J) = f(J): the spectrum of the bipartite chain is symmetric
    assert abs(xy.lnz_exact_infinite(2.0, J=-1.0) - xy.lnz_exact_infinite(2.0)) < 1e-12


def test_trotter_product_is_second_order():
    # SM Sec. F: e^{-tau/2 H_o} e^{-tau H_e} e^{-tau/2 H_o} = e^{-tau H} + O(tau^3)
    from scipy.linalg import expm
    N = 6
    H = xy.hamiltonian_dense(N)
    errs = [np.abs(xy.trotter_dense(N, t) - expm(-t * H)).max() for t in (0.2, 0.1)]
    assert 7.0 < errs[0] / errs[1] < 9.0


@pytest.mark.parametrize("L", [2, 3, 4])
def test_mpo_cell_ring_equals_dense_trotter_operator(L):
    tau = 0.1
    T0 = xy.mpo_cell(tau)
    dense = xy.trotter_dense(2 * L, tau)
    assert np.abs(xy.mpo_ring_dense(T0, L) - dense).max() < 1e-13
    assert abs(xy.mpo_ring_trace(T0, L) / np.trace(dense) - 1) < 1e-13


@pytest.mark.parametrize("L", [2, 3])
def test_untruncated_vertical_merges_equal_dense_powers(L):
    # two untruncated steps: rho(4 tau) on a ring of L cells, against the dense
    # fourth power of the Trotter operator (pins the merge order, the norms and
    # the per-copy bookkeeping)
    tau = 0.1
    fwd = xtrg.xtrg_forward(xy.mpo_cell(tau), 10 ** 6, 2, evaluate=False)
    R = np.linalg.matrix_power(xy.trotter_dense(2 * L, tau), 4)
    assert abs(xtrg.ring_lnz(fwd, L) - math.log(np.trace(R))) < 1e-12


def test_infinite_chain_value_is_the_large_ring_limit():
    fwd = xtrg.xtrg_forward(xy.mpo_cell(0.2), 10 ** 6, 2, evaluate=False)
    L = 4096
    per_cell = xtrg.ring_lnz(fwd, L) / L
    lam = xtrg.dominant(xtrg.transfer_matrix(fwd["T_final"]))[0]
    S = sum(lc / 2.0 ** (j + 1) for j, lc in enumerate(fwd["log_norms"]))
    assert abs(per_cell - (4 * S + math.log(lam))) < 1e-12


@pytest.mark.parametrize("tau", [0.04, 0.02])
def test_untruncated_infinite_chain_against_exact_solution(tau):
    # one untruncated step and the exact final product: rho(4 tau) of the
    # infinite chain, whose Trotter error at beta = 4 tau is O(tau^4) here;
    # also the same value from the large-ring limit of the explicit product
    fwd = xtrg.xtrg_forward(xy.mpo_cell(tau), 10 ** 6, 1)
    beta = 4 * tau
    err = xtrg.lnz_per_site(fwd["lnz"], 2) - xy.lnz_exact_infinite(beta)
    assert abs(err) < 1e-7 * (tau / 0.04) ** 4
    fwd2 = xtrg.xtrg_forward(xy.mpo_cell(tau), 10 ** 6, 2, evaluate=False)
    L = 1 << 14
    assert abs(xtrg.ring_lnz(fwd2, L) / L / 2 - xtrg.lnz_per_site(fwd["lnz"], 2)) < 1e-12


def test_trotter_error_falls_with_tau_at_fixed_beta():
    beta = 0.16
    errs = []
    for tau in (0.02, 0.01):
        n = int(round(math.log2(beta / tau))) - 1
        fwd = xtrg.xtrg_forward(xy.mpo_cell(tau), 32, n)
        errs.append(abs(xtrg.lnz_per_site(fwd["lnz"], n + 1) - xy.lnz_exact_infinite(beta)))
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_truncated_cooling_accuracy_and_monotone_in_d_cut():
    tau = 2.0 ** -10
    T0 = xy.mpo_cell(tau)
    k = 10                      # beta = 2^(k+1) tau = 2
    ex = xy.lnz_exact_infinite(2.0)
    errs = []
    for D in (6, 8, 16):
        fwd = xtrg.xtrg_forward(T0, D, k)
        errs.append(abs(xtrg.lnz_per_site(fwd["lnz"], k + 1) - ex) / ex)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def _fd(f, x, idx, eps):
    xp, xm = x.copy(), x.copy()
    xp[idx] += eps
    xm[idx] -= eps
    return (f(xp) - f(xm)) / (2 * eps)


def test_full_gradient_against_finite_differences_and_euler_identity():
    T0 = xy.mpo_cell(0.05)
    D, n = 6, 3
    fwd = xtrg.xtrg_forward(T0, D, n)
    g = xtrg.xtrg_backward(fwd)
    f = lambda T: xtrg.xtrg_forward(T, D, n, keep=False)["lnz"]
    rng = np.random.default_rng(0)
    for flat in rng.choice(T0.size, 12, replace=False):
        idx = np.unravel_index(flat, T0.shape)
        fd = _fd(f, T0, idx, 1e-6)
        assert abs(fd - g[idx]) < 1e-7 * max(1.0, np.abs(g).max())
    # out(lambda T0) = out(T0) + ln lambda  =>  <T0, d out / d T0> = 1
    assert abs(float(np.sum(T0 * g)) - 1.0) < 1e-11


def test_fixed_w_environments_against_finite_differences():
    T0 = xy.mpo_cell(0.05)
    base = xtrg.xtrg_forward(T0, 6, 3)
    ws = [ck["w"] for ck in base["ckpt"]]
    _, wbars = xtrg.environments(T0, ws)
    rng = np.random.default_rng(1)
    for k in (1, 3):
        w = ws[k - 1]

        def f(wk):
            w2 = list(ws)
            w2[k - 1] = wk
            return xtrg.xtrg_forward(T0, 0, 3, ws=w2, keep=False)["lnz"]

        for flat in rng.choice(w.size, 6, replace=False):
            idx = np.unravel_index(flat, w.shape)
            assert abs(_fd(f, w, idx, 1e-6) - wbars[k - 1][idx]) < 1e-8


def test_seed_scale_is_pinned_by_finite_differences():
    # the finite differences tell the seed (through the exact final product,
    # weight 1/2 in E_n) from one off by the factor 2 of the last level
    T0 = xy.mpo_cell(0.05)
    fwd = xtrg.xtrg_forward(T0, 6, 2)
    g = xtrg.xtrg_backward(fwd)
    f = lambda T: xtrg.xtrg_forward(T, 6, 2, keep=False)["lnz"]
    idx = (0, 0, 0, 0)
    fd = _fd(f, T0, idx, 1e-6)
    assert abs(fd - g[idx]) < 1e-7
    assert abs(fd - 0.5 * g[idx]) > 1e-4


def test_dtrg_cooling_improves_on_scheme_b_and_depth_helps():
    tau = 2.0 ** -10
    T0 = xy.mpo_cell(tau)
    k = 10
    ex = xy.lnz_exact_infinite(2.0)
    r1 = xtrg.dtrg_cooling(T0, 8, k, n_d=1, n_sweeps=1, n_inner=5)
    r2 = xtrg.dtrg_cooling(T0, 8, k, n_d=2, n_sweeps=2, n_inner=5)
    e0 = abs(xtrg.lnz_per_site(r1["lnz_hotrg_steps"][-1], k + 1) - ex)
    e1 = abs(xtrg.lnz_per_site(r1["lnz_steps"][-1], k + 1) - ex)
    e2 = abs(xtrg.lnz_per_site(r2["lnz_steps"][-1], k + 1) - ex)
    assert e1 < e0 and e2 < 0.5 * e1
    for w in r2["ws"]:
        X1, X2, Dp = w.shape
        m = w.reshape(X1 * X2, Dp)
        assert np.abs(m.T @ m - np.eye(Dp)).max() < 1e-12
