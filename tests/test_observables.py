"""Host-side finite differences used for the specific heat (CPU) and the
GPU thermodynamics on a beta grid against the oracle's stored values."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import exact


def test_grid_derivative_is_second_order_exact_on_quadratics():
    from paper_1912_02780_gb300.observables import grid_derivative
    x = np.linspace(0.3, 0.6, 11)
    y = 3 * x ** 2 - 2 * x + 1
    assert np.max(np.abs(grid_derivative(x, y) - (6 * x - 2))) < 1e-12


def test_grid_derivative_matches_onsager_energy_derivative():
    # u = -d(lnZ/N)/dbeta of Onsager's closed form, differentiated on a fine grid
    from paper_1912_02780_gb300.observables import grid_derivative
    b = np.linspace(0.30, 0.36, 13)
    lnz = np.array([exact.onsager_lnz_1d(x) for x in b])
    d = grid_derivative(b, lnz)
    e = 1e-5
    ref = np.array([(exact.onsager_lnz_1d(x + e) - exact.onsager_lnz_1d(x - e)) / (2 * e) for x in b])
    err = np.abs(d - ref)
    assert np.max(err) < 5e-4
    # second order: halving the spacing divides the interior error by about 4
    b2 = np.linspace(0.30, 0.36, 25)
    d2 = grid_derivative(b2, np.array([exact.onsager_lnz_1d(x) for x in b2]))
    ratio = err[6] / abs(d2[12] - ref[6])
    assert 3.0 < ratio < 5.0


@pytest.mark.gpu
def test_ising_grid_against_stored_oracle():
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_grid.json")
    if not os.path.exists(path):
        pytest.skip("golden c2_grid not generated")
    g = json.load(open(path))
    pts = g["points"]
    idx = list(range(0, 64, 9))          # 8 of the 64 grid points
    from paper_1912_02780_gb300.observables import ising_thermodynamics
    betas = np.array([pts[i]["beta"] for i in idx])
    res = ising_thermodynamics(betas, g["d_cut"], g["n_steps"], "bf16x6", split_from_step=7)
    lnz_ref = np.array([pts[i]["lnz"] for i in idx])
    u_ref = -np.array([pts[i]["dlnz_dbeta"] for i in idx])
    df = np.abs(res["lnz"] - lnz_ref) / betas
    du = np.abs(res["u"] - u_ref) / np.abs(u_ref)
    print(f"c2 grid: max |df| = {df.max():.2e}, max rel du = {du.max():.2e}")
    assert df.max() < 1e-9
    assert du.max() < 1e-6


@pytest.mark.gpu
def test_ising_grid_fp64_and_specific_heat_against_stored_oracle():
    """C2 as specified: FP64 on the GPU (Ising, D_cut = 32, 30 steps), forward
    and hand-written adjoint at 8 of the 64 grid points -- four consecutive
    ones around the specific-heat peak next to beta_c, and four spread over
    the grid -- against the oracle's stored ln Z/N and d(ln Z/N)/d beta:
    |df| <= 1e-9 and |du| <= 1e-6 relative.  The specific heat
    c = -beta^2 du/dbeta is compared at the two interior points of the
    consecutive run, both sides by the same central difference of their own
    u (the rule of observables.grid_derivative)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_grid.json")
    if not os.path.exists(path):
        pytest.skip("golden c2_grid not generated")
    g = json.load(open(path))
    pts = g["points"]
    run = [28, 29, 30, 31]                 # beta 0.433 .. 0.448, across beta_c = 0.4407
    idx = [0, 15, 47, 63] + run
    from paper_1912_02780_gb300.observables import ising_thermodynamics
    betas = np.array([pts[i]["beta"] for i in idx])
    res = ising_thermodynamics(betas, g["d_cut"], g["n_steps"], "fp64")
    lnz_ref = np.array([pts[i]["lnz"] for i in idx])
    u_ref = -np.array([pts[i]["dlnz_dbeta"] for i in idx])
    df = np.abs(res["lnz"] - lnz_ref) / betas
    du = np.abs(res["u"] - u_ref) / np.abs(u_ref)
    # specific heat on the consecutive run (positions 4..7 of idx)
    h = pts[1]["beta"] - pts[0]["beta"]
    u_run, u_run_ref, b_run = res["u"][4:], u_ref[4:], betas[4:]
    c = -b_run[1:-1] ** 2 * (u_run[2:] - u_run[:-2]) / (2 * h)
    c_ref = -b_run[1:-1] ** 2 * (u_run_ref[2:] - u_run_ref[:-2]) / (2 * h)
    dc = np.abs(c - c_ref) / np.abs(c_ref)
    print(f"c2 grid fp64: max |df| = {df.max():.2e}, max rel du = {du.max():.2e}, "
          f"c = {c}, max rel dc = {dc.max():.2e}")
    assert df.max() < 1e-9
    assert du.max() < 1e-6
    assert dc.max() < 1e-6
    assert np.all(c > 0)


@pytest.mark.gpu
def test_ising_grid_concurrent_plans_equal_single_plan():
    """Several plans on their own streams (the grid's concurrent mode) give
    every beta the same result as one plan, bit for bit."""
    from paper_1912_02780_gb300.observables import ising_thermodynamics
    betas = np.linspace(0.40, 0.46, 6)
    a = ising_thermodynamics(betas, 16, 16, "bf16x6", split_from_step=5)
    b = ising_thermodynamics(betas, 16, 16, "bf16x6", split_from_step=5, concurrent=3,
                             sm_reserve=16)
    assert np.array_equal(a["lnz"], b["lnz"]) and np.array_equal(a["u"], b["u"])


@pytest.mark.gpu
def test_ising_grid_grouped_forwards_equal_single_plan():
    """The grid in grouped forwards (each stage of a batch of betas one
    tensor-core launch, then each plan's backward) gives every beta the same
    result as one plan, bit for bit, including a last, partial batch."""
    from paper_1912_02780_gb300.observables import ising_thermodynamics
    betas = np.linspace(0.40, 0.46, 7)
    a = ising_thermodynamics(betas, 16, 16, "bf16x6", split_from_step=5)
    b = ising_thermodynamics(betas, 16, 16, "bf16x6", split_from_step=5, grouped=3)
    assert np.array_equal(a["lnz"], b["lnz"]) and np.array_equal(a["u"], b["u"])
