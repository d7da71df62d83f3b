"""Pins of the differentiable-TRG oracle (oracle/dtrg.py): the MERA update is
the trace maximiser, the environments are the derivatives of ln Z / N, a
sweep is a no-op where nothing is truncated, the sweeps improve on HOTRG
(main text Fig. 2: dTRG below HOTRG off criticality) and converge to the
polar fixed point."""
import numpy as np

from oracle import dtrg, exact, hotrg, ising


def test_mera_update_is_the_trace_maximiser():
    rng = np.random.default_rng(5)
    E = rng.standard_normal((6, 6, 9))
    w = dtrg.mera_update(E)
    W, M = w.reshape(36, 9), E.reshape(36, 9)
    assert np.max(np.abs(W.T @ W - np.eye(9))) < 1e-13
    best = float(np.sum(M * W))
    assert abs(best - np.sum(np.linalg.svd(M, compute_uv=False))) < 1e-12 * best
    for _ in range(200):                      # no other isometry does better
        Q, _ = np.linalg.qr(rng.standard_normal((36, 9)))
        assert float(np.sum(M * Q)) < best


def test_environment_is_the_derivative():
    T0 = ising.ising_T0(0.42, 1.0, 0.02)
    base = hotrg.hotrg_forward(T0, 4, 6)
    ws = [ck["w"] for ck in base["ckpt"]]
    lnz, wb = dtrg.environments(T0, ws)
    assert abs(lnz - base["lnz"]) < 1e-14     # same network as HOTRG's
    rng = np.random.default_rng(0)
    eps = 1e-6
    for k in (1, 3, 6):
        d = rng.standard_normal(ws[k - 1].shape)
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[k - 1] += eps * d
        wm[k - 1] -= eps * d
        fd = (dtrg.forward_fixed_w(T0, wp)["lnz"] - dtrg.forward_fixed_w(T0, wm)["lnz"]) / (2 * eps)
        an = float(np.sum(wb[k - 1] * d))
        assert abs(fd - an) < 1e-7 * abs(an)


def test_untruncated_sweep_leaves_lnz_exact():
    beta, h, n = 0.41, 0.03, 4
    T0 = ising.ising_T0(beta, 1.0, h)
    r = dtrg.dtrg_sweeps(T0, 10 ** 6, n, n_sweeps=1, n_inner=1)
    Lx, Ly = 2 ** (n // 2), 2 ** ((n + 1) // 2)
    ref = exact.torus_lnz(T0, Lx, Ly) / (Lx * Ly)
    assert abs(r["lnz_hotrg"] - ref) < 1e-12
    assert abs(r["lnz_final"] - ref) < 1e-12


def test_dtrg_improves_on_hotrg_off_critical():
    beta = 0.40
    T0 = ising.ising_T0(beta)
    r = dtrg.dtrg_sweeps(T0, 6, 16, n_sweeps=1, n_inner=2)
    ons = exact.onsager_lnz(beta)
    err_h, err_d = abs(r["lnz_hotrg"] - ons), abs(r["lnz_final"] - ons)
    assert r["lnz_final"] > r["lnz_hotrg"]    # the sweep raised Z
    assert err_d < err_h / 3                   # 1.25e-5 -> 2.9e-6 measured


def test_sweeps_reach_the_polar_fixed_point():
    T0 = ising.ising_T0(0.40)
    r = dtrg.dtrg_sweeps(T0, 6, 16, n_sweeps=4, n_inner=2)
    _, wb = dtrg.environments(T0, r["ws"])
    for k in range(1, 9):
        w, E = r["ws"][k - 1], wb[k - 1]
        N, D = w.shape[0] * w.shape[1], w.shape[2]
        M = w.reshape(N, D).T @ E.reshape(N, D)   # w = polar(E)  <=>  w^T E symmetric
        assert np.max(np.abs(M - M.T)) < 1e-5 * np.max(np.abs(M))
