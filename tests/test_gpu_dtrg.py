"""Differentiable-TRG sweeps on the GPU against the oracle (oracle/dtrg.py):
the isometry environments d(ln Z/N)/d w_k of the backward, and whole sweeps
of MERA updates (cuSOLVER SVD + FP64 GEMM through hotrg_mera_update)."""
import numpy as np
import pytest

import synth
from oracle import dtrg as odtrg
from oracle import hotrg, ising

pytestmark = pytest.mark.gpu
hot = pytest.importorskip("paper_1912_02780_gb300")


def test_isometry_adjoints_match_oracle():
    """d(ln Z/N)/d w_k of the GPU backward (fixed w) against the oracle's
    backward of the same network: the oracle is given the GPU's isometries,
    so the comparison is free of the eigenvector gauge (degenerate spectra
    leave the isometries themselves undetermined)."""
    T0 = synth.random_symmetric_T0(1, 4)
    with hot.Plan(4, 8, 8, "fp64", fixed_w_grad=True) as p:
        lnz, _, _ = p.forward_tensor(T0)
        p.backward()
        ws = p.isometries()
        wb = p.isometry_adjoints()
    fwd = odtrg.forward_fixed_w(T0, ws)
    assert abs(fwd["lnz"] - lnz) < 1e-12
    _, wb_ref = hotrg.hotrg_backward(fwd, fixed_w=True, return_wbar=True)
    for k in range(8):
        W = ws[k].reshape(-1, ws[k].shape[2])
        assert np.max(np.abs(W.T @ W - np.eye(W.shape[1]))) < 1e-12
        assert np.max(np.abs(wb[k] - wb_ref[k])) < 1e-10 * np.max(np.abs(wb_ref[k]))


def test_dtrg_sweep_fp64_matches_oracle():
    """One sweep of two MERA updates per layer (Ising beta = 0.40, D = 6,
    16 steps): ln Z / N before and after agrees with the oracle's sweep to
    rounding, Z grew, and the updated isometries are orthonormal and give
    that ln Z / N in the oracle's forward."""
    beta = 0.40
    ref = odtrg.dtrg_sweeps(ising.ising_T0(beta), 6, 16, n_sweeps=1, n_inner=2)
    from paper_1912_02780_gb300.dtrg import dtrg_sweeps
    r = dtrg_sweeps(2, 6, 16, n_sweeps=1, n_inner=2, beta=beta)
    print(f"dtrg fp64: hotrg {r['lnz_hotrg'] - ref['lnz_hotrg']:.2e}, "
          f"sweep {r['lnz_final'] - ref['lnz_final']:.2e}")
    assert abs(r["lnz_hotrg"] - ref["lnz_hotrg"]) < 1e-12
    assert abs(r["lnz_final"] - ref["lnz_final"]) < 1e-11
    assert r["lnz_final"] > r["lnz_hotrg"]
    for w in r["isometries"]:
        W = w.reshape(-1, w.shape[2])
        assert np.max(np.abs(W.T @ W - np.eye(W.shape[1]))) < 1e-12
    assert abs(odtrg.forward_fixed_w(ising.ising_T0(beta), r["isometries"])["lnz"]
               - r["lnz_final"]) < 1e-12


def test_dtrg_sweep_split_close_to_oracle():
    """Split precision (BF16X6 from step 3, D = 16): the environments carry
    the split backward's ~1e-7 relative error into the MERA updates, so the
    swept ln Z / N is held to 1e-8 (the HOTRG start to 1e-9)."""
    T0 = synth.random_symmetric_T0(0, 4)
    ref = odtrg.dtrg_sweeps(T0, 16, 6, n_sweeps=1, n_inner=1)
    from paper_1912_02780_gb300.dtrg import dtrg_sweeps
    r = dtrg_sweeps(4, 16, 6, n_sweeps=1, n_inner=1, T0=T0, precision="bf16x6",
                    split_from_step=3)
    err = abs(r["lnz_final"] - ref["lnz_final"])
    print(f"dtrg bf16x6 D=16: |dlnz| = {err:.2e} (HOTRG {abs(r['lnz_hotrg'] - ref['lnz_hotrg']):.2e})")
    assert abs(r["lnz_hotrg"] - ref["lnz_hotrg"]) < 1e-9
    assert err < 1e-8


def test_w_given_plan_needs_isometries_first():
    with hot.Plan(2, 6, 6, "fp64", fixed_w_grad=True, w_given=True) as p:
        with pytest.raises(hot.HotrgError) as e:
            p.forward_ising(0.4)
        assert e.value.status == 7                       # HOTRG_ESTATE
        with pytest.raises(hot.HotrgError) as e2:
            p.mera_update(1)
        assert e2.value.status == 7


def test_dtrg_improves_on_hotrg_near_criticality():
    """Main text Fig. 2 (shape only; the plotted values are not available):
    free-energy error against Onsager of HOTRG and of dTRG (one sweep, three
    MERA updates per layer) at D_cut = 24, 30 steps (2^30 sites, finite-size
    terms far below these errors off criticality), split precision."""
    from oracle import exact
    from paper_1912_02780_gb300.dtrg import dtrg_sweeps
    rows = []
    for beta in (0.42, float(synth.BETA_C), 0.46):
        r = dtrg_sweeps(2, 24, 30, n_sweeps=1, n_inner=3, beta=beta, precision="bf16x6",
                        split_from_step=5)
        ons = exact.onsager_lnz(beta)
        e_h = abs(r["lnz_hotrg"] - ons) / abs(ons)
        e_d = abs(r["lnz_final"] - ons) / abs(ons)
        rows.append((beta, e_h, e_d))
        print(f"beta = {beta:.6f}: |df/f| HOTRG {e_h:.3e}, dTRG {e_d:.3e}")
    for beta, e_h, e_d in rows:
        if abs(beta - synth.BETA_C) > 1e-3:
            assert e_d < e_h


@pytest.mark.parametrize("layers", [None, [3]])
def test_lbfgs_sweeps_against_oracle(layers):
    """L-BFGS in the exponential parametrisation (SM Sec. D) on the GPU against
    the oracle's iterates, layer by layer, on the Ising network at beta = 0.40."""
    from oracle import ising, lbfgs as olb
    from paper_1912_02780_gb300 import dtrg as gd
    beta, D, n = 0.40, 6, 8
    n_iter = 5 if layers is None else 30
    T0 = ising.ising_T0(beta, 1.0, 0.0)
    ref = olb.lbfgs_sweeps(T0, D, n, n_sweeps=1, n_iter=n_iter, layers=layers)
    got = gd.lbfgs_sweeps(2, D, n, n_sweeps=1, n_iter=n_iter, beta=beta, layers=layers)
    assert abs(got["lnz_hotrg"] - ref["lnz_hotrg"]) < 1e-13
    for a, b in zip(got["layer_hist"], ref["layer_hist"]):
        assert len(a) == len(b)
        assert np.abs(np.asarray(a) - np.asarray(b)).max() < 1e-12
    assert abs(got["lnz"][-1] - ref["lnz"][-1]) < 1e-12
    assert got["lnz"][-1] > got["lnz_hotrg"]
    for w in got["isometries"]:
        X1, X2, Dp = w.shape
        m = w.reshape(X1 * X2, Dp)
        assert np.abs(m.T @ m - np.eye(Dp)).max() < 1e-12
