"""Scheme (b) on the GPU (vertical-only coarse-graining of the XY chain's
density-matrix MPO, main text Fig. 1b) against the FP64 oracle
(oracle/xtrg.py, oracle/xy.py): forward at every depth, full gradient,
fixed-w environments, differentiable-TRG cooling, and the exact solution."""
import math
import warnings

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
warnings.filterwarnings("ignore", message=".*roundoff error.*")


@pytest.fixture(scope="module")
def hot():
    import paper_1912_02780_gb300 as h
    return h


def _f_site(out_k, k, tau):
    beta = tau * 2.0 ** (k + 1)
    return -(2.0 ** k) * out_k / beta


# Bond dimensions whose cuts are not degenerate: the XY chain conserves S^z,
# so the Gram spectra have exactly degenerate pairs, and where the cut falls
# inside one the truncation depends on rounding (at D = 16 the oracle itself
# moves by 5e-8 in f under an orthogonal change of the bond basis of T0; at
# D = 12 and 24 by below 1e-11).
@pytest.mark.parametrize("d_cut", [12, 24])
def test_forward_every_depth_against_oracle(hot, d_cut):
    from oracle import xtrg, xy
    tau, n = 2.0 ** -8, 10
    T0 = xy.mpo_cell(tau)
    ref = xtrg.xtrg_forward(T0, d_cut, n)["lnz_steps"]
    with hot.Plan(4, d_cut, n, want_grad=False, scheme=1, chain_steps=True) as p:
        # the oracle's cell tensor, and the one the library builds on the device
        # (another bond gauge of the same operator: the same Z)
        p.forward_tensor(T0)
        got_t = p.chain_lnz_steps()
        lnz_xy, ln = p.forward_xy(tau)
        got_xy = p.chain_lnz_steps()
    assert lnz_xy == got_xy[-1]
    for k in range(1, n + 1):
        for got in (got_t, got_xy):
            assert abs(_f_site(got[k - 1], k, tau) - _f_site(ref[k - 1], k, tau)) < 1e-9


def test_last_depth_only_equals_every_depth(hot):
    from oracle import xy
    tau, n = 2.0 ** -8, 8
    with hot.Plan(4, 16, n, want_grad=False, scheme=1, chain_steps=True) as p:
        a = p.forward_xy(tau)[0]
    with hot.Plan(4, 16, n, want_grad=False, scheme=1) as p:
        b = p.forward_xy(tau)[0]
        steps = p.chain_lnz_steps()
    assert a == b
    assert np.all(np.isnan(steps[:-1])) and steps[-1] == b


def test_subspace_eigensolver_forward(hot):
    from oracle import xtrg, xy
    tau, n, D = 2.0 ** -8, 10, 24
    T0 = xy.mpo_cell(tau)
    ref = xtrg.xtrg_forward(T0, D, n)["lnz"]
    with hot.Plan(4, D, n, want_grad=False, scheme=1, eigh_mode=1, eigh_power_iters=2) as p:
        got = p.forward_tensor(T0)[0]
    assert abs(_f_site(got, n, tau) - _f_site(ref, n, tau)) < 1e-9


def test_full_gradient_against_oracle(hot):
    from oracle import xtrg, xy
    tau, D, n = 0.05, 10, 4          # relative cut gaps >= 1e-7
    T0 = xy.mpo_cell(tau)
    fwd = xtrg.xtrg_forward(T0, D, n)
    g_ref = xtrg.xtrg_backward(fwd)
    with hot.Plan(4, D, n, want_grad=True, scheme=1) as p:
        lnz = p.forward_tensor(T0)[0]
        g = p.backward()
    assert abs(lnz - fwd["lnz"]) < 1e-13
    assert np.abs(g - g_ref).max() / np.abs(g_ref).max() < 1e-8
    assert abs(float(np.sum(T0 * g)) - 1.0) < 1e-10     # <T0, d out / d T0> = 1


def test_fixed_w_environments_against_oracle(hot):
    from oracle import xtrg, xy
    tau, D, n = 0.05, 10, 4
    T0 = xy.mpo_cell(tau)
    ws = [ck["w"] for ck in xtrg.xtrg_forward(T0, D, n)["ckpt"]]
    lnz_ref, wb_ref = xtrg.environments(T0, ws)
    with hot.Plan(4, D, n, want_grad=True, fixed_w_grad=True, w_given=True, scheme=1) as p:
        p.set_isometries(ws)
        lnz = p.forward_tensor(T0)[0]
        p.backward()
        wb = p.isometry_adjoints()
    assert abs(lnz - lnz_ref) < 1e-13
    for a, b in zip(wb, wb_ref):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_given_steps_grow_the_network_like_hotrg(hot):
    from oracle import xy
    tau, D, n = 2.0 ** -8, 12, 6
    with hot.Plan(4, D, n, want_grad=False, scheme=1) as p:
        ref = p.forward_xy(tau)[0]
    with hot.Plan(4, D, n, want_grad=True, fixed_w_grad=True, w_given=True, scheme=1) as p:
        with pytest.raises(hot.HotrgError):
            p.forward_xy(tau)                 # no isometries defined yet
        vals = []
        for k in range(1, n + 1):
            p.set_steps(k)
            p.set_given_steps(k - 1)
            vals.append(p.forward_xy(tau)[0])  # layer k formed from its Gram matrix
        p.set_given_steps(n)
        again = p.forward_xy(tau)[0]           # all layers now given
    assert abs(vals[-1] - ref) < 1e-14 and abs(again - ref) < 1e-14


def test_dtrg_cooling_against_oracle_and_exact(hot):
    from oracle import xtrg, xy
    from paper_1912_02780_gb300 import xtrg as gx
    tau, D, n = 2.0 ** -10, 10, 10
    ref = xtrg.dtrg_cooling(xy.mpo_cell(tau), D, n, n_d=2, n_sweeps=2, n_inner=5)
    got = gx.cooling(tau, D, n, n_d=2, n_sweeps=2, n_inner=5)
    for k in range(1, n + 1):
        assert abs(_f_site(got["lnz_copy"][k - 1], k, tau) -
                   _f_site(ref["lnz_steps"][k - 1], k, tau)) < 1e-9
    plain = gx.cooling(tau, D, n)
    ex = -xy.lnz_exact_infinite(2.0) / 2.0
    assert abs(got["beta"][-1] - 2.0) < 1e-15
    assert abs(got["f"][-1] - ex) < abs(plain["f"][-1] - ex)


def test_invalid_arguments(hot):
    with hot.Plan(2, 8, 4, want_grad=False) as p:
        with pytest.raises(hot.HotrgError):
            p.forward_xy(0.01)                # needs scheme 1 and d0 = 4
        with pytest.raises(hot.HotrgError):
            p.chain_lnz_steps()
    with hot.Plan(4, 8, 4, want_grad=False, scheme=1) as p:
        with pytest.raises(hot.HotrgError):
            p.forward_xy(-1.0)
        with pytest.raises(hot.HotrgError):
            p.set_given_steps(1)              # not a w_given plan
