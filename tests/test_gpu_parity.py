"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path: the same algorithm in the same precision, so results agree to
rounding (ln Z / N to 1e-12, gradients to 1e-9 relative).  Split tensor-core
path: errors are bounded by the split precision and reported; the tolerances
below follow from the per-product error of the planes and the 2^-k weight of
step k in ln Z / N.
"""
import math

import numpy as np
import pytest

import synth
from oracle import exact, hotrg, ising

hot = pytest.importorskip("paper_1912_02780_gb300")
pytestmark = pytest.mark.gpu


def torus_dims(n):
    return 2 ** (n // 2), 2 ** ((n + 1) // 2)


@pytest.mark.parametrize("M,N,K", [(64, 48, 40), (200, 300, 136), (1, 7, 8)])
def test_gemm_f64_kernel(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A, B = rng.standard_normal((M, K)), rng.standard_normal((N, K))
    C = hot.gemm_f64_check(A, B)
    assert np.max(np.abs(C - A @ B.T)) < 1e-12 * np.max(np.abs(A) @ np.abs(B).T)


@pytest.mark.parametrize("planes,kchunk", [(2, 0), (3, 0), (3, 2), (2, 3)])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 520), (1000, 72, 4096), (5, 700, 8)])
def test_gemm_split_kernel(planes, kchunk, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A, B = rng.standard_normal((M, K)), rng.standard_normal((N, K))
    C = hot.gemm_split_check(A, B, planes=planes, kchunk=kchunk)
    scale = np.abs(A) @ np.abs(B).T
    err = np.max(np.abs(C - A @ B.T) / scale)
    bound = {2: 3e-5, 3: 4e-6}[planes]
    assert err < bound, err


def test_forward_fp64_ising_C1():
    beta = 0.44
    ref = hotrg.hotrg_forward(ising.ising_T0(beta), 8, 20, keep=False)
    with hot.Plan(2, 8, 20, "fp64", want_grad=False) as p:
        lnz, ln, sign = p.forward_ising(beta, 1.0, 0.0)
    assert abs(lnz - ref["lnz"]) < 1e-12
    assert np.max(np.abs(ln - np.array(ref["log_norms"]))) < 1e-10
    assert sign == ref["trace_sign"]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_forward_fp64_untruncated_equals_exact_torus(n):
    beta, h = 0.41, 0.03
    T0 = ising.ising_T0(beta, 1.0, h)
    Lx, Ly = torus_dims(n)
    with hot.Plan(2, 10 ** 6, n, "fp64", want_grad=False) as p:
        lnz, _, _ = p.forward_tensor(T0)
    assert abs(lnz - exact.torus_lnz(T0, Lx, Ly) / (Lx * Ly)) < 1e-12


@pytest.mark.parametrize("seed,d_cut,n", [(0, 16, 10), (3, 12, 9)])
def test_forward_fp64_random_tensor(seed, d_cut, n):
    T0 = synth.random_symmetric_T0(seed, 4)
    ref = hotrg.hotrg_forward(T0, d_cut, n, keep=False)
    with hot.Plan(4, d_cut, n, "fp64", want_grad=False) as p:
        lnz, ln, sign = p.forward_tensor(T0)
    assert abs(lnz - ref["lnz"]) < 1e-12
    assert np.max(np.abs(ln - np.array(ref["log_norms"]))) < 1e-9


@pytest.mark.parametrize("fixed_w", [False, True])
def test_backward_fp64_ising_C1(fixed_w):
    beta = 0.44
    f = hotrg.hotrg_forward(ising.ising_T0(beta), 8, 20)
    g_ref = hotrg.hotrg_backward(f, fixed_w=fixed_w)
    db_ref = float(np.sum(g_ref * ising.ising_dT0_dbeta(beta)))
    with hot.Plan(2, 8, 20, "fp64", fixed_w_grad=fixed_w) as p:
        p.forward_ising(beta, 1.0, 0.0)
        g, db = p.backward(want_dbeta=True)
    assert np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref)) < 1e-9
    assert abs(db - db_ref) / abs(db_ref) < 1e-9


def test_backward_fp64_random_tensor_and_euler():
    T0 = synth.random_symmetric_T0(1, 4)
    f = hotrg.hotrg_forward(T0, 12, 8)
    g_ref = hotrg.hotrg_backward(f)
    with hot.Plan(4, 12, 8, "fp64") as p:
        p.forward_tensor(T0)
        g = p.backward()
    assert np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref)) < 1e-9
    assert abs(np.sum(g * T0) - 1.0) < 1e-11


@pytest.mark.parametrize("precision,tol", [("bf16x3", 5e-6), ("bf16x6", 1e-6)])
@pytest.mark.parametrize("d_cut", [16, 32])
def test_forward_split_random_tensor(precision, tol, d_cut):
    T0 = synth.random_symmetric_T0(0, 4)
    n = 14
    ref = hotrg.hotrg_forward(T0, d_cut, n, keep=False)
    with hot.Plan(4, d_cut, n, precision, split_from_step=1, want_grad=False) as p:
        lnz, ln, _ = p.forward_tensor(T0)
        _, _, is_split = p.diagnostics()
    assert is_split.sum() > 0
    err = abs(lnz - ref["lnz"])
    print(f"{precision} D={d_cut}: |dlnz| = {err:.3e}")
    assert err < tol
