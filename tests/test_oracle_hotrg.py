"""Pins of the oracle HOTRG forward and backward (oracle/hotrg.py).

What fixes each function independently of itself:
* untruncated HOTRG (D_cut >= every X^2) is an exact contraction, so it must
  equal the exact transfer-matrix torus (and brute-force enumeration) on the
  2^floor(n/2) x 2^ceil(n/2) torus -- with a random T0 that is not
  rotation-symmetric this also pins the x/y alternation;
* untruncated Z does not depend on w at all (any orthogonal w);
* the isometry is orthonormal and the Gram matrix is PSD;
* truncated HOTRG converges to Onsager's free energy with growing D_cut;
* limits: beta = 0 gives ln 2, f(h) = f(-h), deep ordered phase;
* Euler identity <T0, d(lnZ/N)/dT0> = 1 for any truncation (Z is
  homogeneous of degree N in T0 and w is scale invariant);
* gradients against central finite differences of the forward (full mode)
  and of the forward with the isometries frozen (fixed-w mode);
* untruncated beta derivative against the exact enumerated energy.
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg, ising
import synth


def torus_dims(n):
    return 2 ** (n // 2), 2 ** ((n + 1) // 2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.05), (0.6, 0.01)])
def test_untruncated_ising_equals_exact_torus(n, beta, h):
    T0 = ising.ising_T0(beta, 1.0, h)
    f = hotrg.hotrg_forward(T0, 10 ** 6, n, keep=False)
    Lx, Ly = torus_dims(n)
    ref = exact.torus_lnz(T0, Lx, Ly) / (Lx * Ly)
    assert abs(f["lnz"] - ref) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4])
def test_untruncated_ising_equals_bruteforce(n):
    beta, h = 0.41, 0.03
    f = hotrg.hotrg_forward(ising.ising_T0(beta, 1.0, h), 10 ** 6, n, keep=False)
    Lx, Ly = torus_dims(n)
    assert abs(f["lnz"] - exact.bruteforce(Lx, Ly, beta, 1.0, h)[0]) < 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_untruncated_random_tensor_pins_orientation(seed, n):
    T0 = synth.random_symmetric_T0(seed, 4)
    # make it clearly anisotropic so that a wrong x/y alternation shows
    T0 = T0 + 0.3 * np.einsum("l,r,u,d->lrud", *(np.arange(4.0) - 1.0 for _ in range(2)), np.ones(4), np.ones(4))
    f = hotrg.hotrg_forward(T0, 10 ** 6, n, keep=False)
    Lx, Ly = torus_dims(n)
    ref = exact.torus_lnz(T0, Lx, Ly) / (Lx * Ly)
    swapped = exact.torus_lnz(T0, Ly, Lx) / (Lx * Ly)
    assert abs(f["lnz"] - ref) < 1e-12
    if Lx != Ly:
        assert abs(swapped - ref) > 1e-6     # the pin can tell the two tori apart


def test_untruncated_independent_of_isometry():
    T0 = ising.ising_T0(0.47, 1.0, 0.02)
    rng = np.random.default_rng(5)

    def random_w(k, X, Dp, lam, U):
        q, _ = np.linalg.qr(rng.standard_normal((X * X, X * X)))
        return q.reshape(X, X, X * X)

    a = hotrg.hotrg_forward(T0, 10 ** 6, 4, keep=False)["lnz"]
    b = hotrg.hotrg_forward(T0, 10 ** 6, 4, keep=False, w_override=random_w)["lnz"]
    assert abs(a - b) < 1e-13


def test_isometry_orthonormal_and_gram_psd():
    f = hotrg.hotrg_forward(synth.random_symmetric_T0(3, 4), 12, 8)
    for ck in f["ckpt"]:
        w = ck["w"].reshape(-1, ck["Dp"])
        assert np.max(np.abs(w.T @ w - np.eye(ck["Dp"]))) < 1e-13
        assert ck["lam"][-1] >= -1e-12 * ck["lam"][0]
        assert np.all(np.diff(ck["lam"]) <= 1e-12 * ck["lam"][0])


def test_gram_is_merged_pair_outer_product():
    # G = M M^T with M[(x1 x2), (x1' x2' y y')] = sum_j T[x1,x1',y,j] T[x2,x2',j,y']
    rng = np.random.default_rng(1)
    T = rng.standard_normal((3, 3, 2, 2))
    M = np.einsum("aiyj,bkjz->abikyz", T, T).reshape(9, -1)
    assert np.allclose(hotrg.gram(T), M @ M.T, rtol=1e-13, atol=1e-13)


def test_step_matches_one_shot_einsum():
    rng = np.random.default_rng(2)
    T = rng.standard_normal((3, 3, 4, 4))
    w = np.linalg.qr(rng.standard_normal((9, 9)))[0][:, :5].reshape(3, 3, 5)
    ref = np.einsum("aiyj,bkjz,abA,ikB->AByz", T, T, w, w)
    assert np.allclose(hotrg.hotrg_step(T, w), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.slow
@pytest.mark.parametrize("beta", [0.30, 0.60])
def test_converges_to_onsager_off_critical(beta):
    # 2^12 x 2^12 torus: finite-size effects are far below the truncation error
    ons = exact.onsager_lnz_1d(beta)
    errs = [abs(hotrg.hotrg_forward(ising.ising_T0(beta), d, 24, keep=False)["lnz"] - ons)
            for d in (4, 8, 12)]
    assert errs[2] < errs[0]
    assert errs[2] < 1e-7


@pytest.mark.slow
def test_near_critical_error_at_truncation_level():
    ons = exact.onsager_lnz_1d(synth.BETA_C)
    f = hotrg.hotrg_forward(ising.ising_T0(synth.BETA_C), 12, 24, keep=False)
    assert abs(f["lnz"] - ons) < 5e-4


def test_limits():
    assert abs(hotrg.hotrg_forward(ising.ising_T0(0.0, 1.0, 0.0), 8, 12, keep=False)["lnz"] - math.log(2)) < 1e-14
    a = hotrg.hotrg_forward(ising.ising_T0(0.45, 1.0, 0.03), 8, 12, keep=False)["lnz"]
    b = hotrg.hotrg_forward(ising.ising_T0(0.45, 1.0, -0.03), 8, 12, keep=False)["lnz"]
    assert abs(a - b) < 1e-13
    beta, h = 1.2, 0.02
    deep = hotrg.hotrg_forward(ising.ising_T0(beta, 1.0, h), 8, 16, keep=False)["lnz"]
    assert abs(deep - beta * (2 + h)) < 10 * math.exp(-8 * beta)


def grad_full(T0, d_cut, n, **kw):
    f = hotrg.hotrg_forward(T0, d_cut, n)
    return f, hotrg.hotrg_backward(f, **kw)


@pytest.mark.parametrize("fixed_w", [False, True])
def test_euler_identity(fixed_w):
    T0 = synth.random_symmetric_T0(0, 4)
    f, g = grad_full(T0, 10, 10, fixed_w=fixed_w)
    assert abs(np.sum(T0 * g) - 1.0) < 1e-12


def test_beta_gradient_matches_finite_differences_C1():
    beta, e = 0.44, 1e-5
    f, g = grad_full(ising.ising_T0(beta), 8, 20)
    db = float(np.sum(g * ising.ising_dT0_dbeta(beta)))
    fp = hotrg.hotrg_forward(ising.ising_T0(beta + e), 8, 20, keep=False)["lnz"]
    fm = hotrg.hotrg_forward(ising.ising_T0(beta - e), 8, 20, keep=False)["lnz"]
    fd = (fp - fm) / (2 * e)
    assert abs(db - fd) / abs(fd) < 1e-7


@pytest.mark.parametrize("seed,d_cut,n", [(0, 6, 6), (1, 9, 7)])
def test_tensor_gradient_matches_finite_differences(seed, d_cut, n):
    T0 = synth.random_symmetric_T0(seed, 3)
    f, g = grad_full(T0, d_cut, n)
    e = 1e-6
    fd = np.zeros_like(T0)
    rng = np.random.default_rng(seed)
    entries = [tuple(int(v) for v in rng.integers(0, 3, size=4)) for _ in range(12)]
    for idx in entries:
        tp, tm = T0.copy(), T0.copy()
        tp[idx] += e
        tm[idx] -= e
        fd[idx] = (hotrg.hotrg_forward(tp, d_cut, n, keep=False)["lnz"]
                   - hotrg.hotrg_forward(tm, d_cut, n, keep=False)["lnz"]) / (2 * e)
    sel = tuple(np.array(entries).T)
    assert np.max(np.abs(g[sel] - fd[sel])) / np.max(np.abs(g)) < 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("seed,d_cut,n", [(0, 6, 6), (1, 9, 7)])
def test_tensor_gradient_matches_finite_differences_all_entries(seed, d_cut, n):
    """The same pin on every one of the 81 entries of T0 (central differences,
    eps = 1e-6, FD error ~1e-10 relative)."""
    T0 = synth.random_symmetric_T0(seed, 3)
    f, g = grad_full(T0, d_cut, n)
    e = 1e-6
    fd = np.zeros_like(T0)
    for idx in np.ndindex(T0.shape):
        tp, tm = T0.copy(), T0.copy()
        tp[idx] += e
        tm[idx] -= e
        fd[idx] = (hotrg.hotrg_forward(tp, d_cut, n, keep=False)["lnz"]
                   - hotrg.hotrg_forward(tm, d_cut, n, keep=False)["lnz"]) / (2 * e)
    assert np.max(np.abs(g - fd)) / np.max(np.abs(fd)) < 1e-6


@pytest.mark.slow
def test_near_critical_error_at_truncation_level_d16_n30():
    """Onsager at beta_c on the 2^15 x 2^15 torus (n = 30, finite-size terms
    ~1/L^2 far below the truncation error) with D_cut = 16: within 1e-4."""
    ons = exact.onsager_lnz_1d(synth.BETA_C)
    f = hotrg.hotrg_forward(ising.ising_T0(synth.BETA_C), 16, 30, keep=False)
    assert abs(f["lnz"] - ons) < 1e-4


@pytest.mark.slow
@pytest.mark.parametrize("beta", [0.30, 0.60])
def test_converges_to_onsager_off_critical_d16_n30(beta):
    """Off criticality the error falls with D_cut (4, 8, 16) on the 2^15 x
    2^15 torus and is below 1e-7 at D_cut = 16."""
    ons = exact.onsager_lnz_1d(beta)
    errs = [abs(hotrg.hotrg_forward(ising.ising_T0(beta), d, 30, keep=False)["lnz"] - ons)
            for d in (4, 8, 16)]
    assert errs[2] < errs[0]
    assert errs[2] < 1e-7


def test_fixed_w_gradient_matches_frozen_isometry_differences():
    T0 = synth.random_symmetric_T0(4, 3)
    d_cut, n = 6, 6
    f, g = grad_full(T0, d_cut, n, fixed_w=True)
    ws = [ck["w"] for ck in f["ckpt"]]

    def frozen(k, X, Dp, lam, U):
        return ws[k - 1]

    e = 1e-6
    fd = np.zeros_like(T0)
    for idx in np.ndindex(T0.shape):
        tp, tm = T0.copy(), T0.copy()
        tp[idx] += e
        tm[idx] -= e
        fd[idx] = (hotrg.hotrg_forward(tp, d_cut, n, keep=False, w_override=frozen)["lnz"]
                   - hotrg.hotrg_forward(tm, d_cut, n, keep=False, w_override=frozen)["lnz"]) / (2 * e)
    assert np.max(np.abs(g - fd)) / np.max(np.abs(fd)) < 1e-6
    full = hotrg.hotrg_backward(f)
    assert np.max(np.abs(full - g)) > 1e-6   # truncation makes the two modes differ


@pytest.mark.parametrize("n", [2, 3, 4])
def test_untruncated_beta_gradient_equals_exact_energy(n):
    beta, h = 0.39, 0.04
    T0 = ising.ising_T0(beta, 1.0, h)
    f = hotrg.hotrg_forward(T0, 10 ** 6, n)
    g_full = hotrg.hotrg_backward(f)
    g_fix = hotrg.hotrg_backward(f, fixed_w=True)
    assert np.max(np.abs(g_full - g_fix)) < 1e-13
    Lx, Ly = torus_dims(n)
    db = float(np.sum(g_full * ising.ising_dT0_dbeta(beta, 1.0, h)))
    assert abs(db - exact.bruteforce(Lx, Ly, beta, 1.0, h)[1]) < 1e-12


def test_w_gradient_matches_finite_differences():
    # d(lnZ/N)/dw_k with every isometry frozen (main-text Eq. (1): the adjoint of w)
    T0 = synth.random_symmetric_T0(2, 3)
    d_cut, n, kk = 6, 5, 3
    f = hotrg.hotrg_forward(T0, d_cut, n)
    _, wbars = hotrg.hotrg_backward(f, fixed_w=True, return_wbar=True)
    ws = [ck["w"].copy() for ck in f["ckpt"]]
    e = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(5):
        idx = tuple(rng.integers(0, s) for s in ws[kk - 1].shape)
        vals = []
        for sgn in (1, -1):
            wk = [w.copy() for w in ws]
            wk[kk - 1][idx] += sgn * e
            vals.append(hotrg.hotrg_forward(T0, d_cut, n, keep=False,
                                            w_override=lambda k, X, Dp, lam, U: wk[k - 1])["lnz"])
        fd = (vals[0] - vals[1]) / (2 * e)
        assert abs(wbars[kk - 1][idx] - fd) < 1e-8 * max(1.0, abs(fd))


# ---- w_rule = 1: the isometry from the side with the smaller truncation error

def test_w_rule_1_equals_left_rule_on_reflection_symmetric_tensors():
    import synth
    for T0 in (ising.ising_T0(0.44, 1.0, 0.0), synth.random_symmetric_T0(0, 4)):
        a = hotrg.hotrg_forward(T0, 6, 6)
        b = hotrg.hotrg_forward(T0, 6, 6, w_rule=1)
        assert a["lnz"] == b["lnz"]
        assert all(ck["side"] == 0 for ck in b["ckpt"])


def test_w_rule_1_takes_the_smaller_truncation_error_on_each_step():
    import synth
    T0 = synth.random_T0(3, 3)
    fwd = hotrg.hotrg_forward(T0, 5, 6, w_rule=1)
    sides = []
    for ck in fwd["ckpt"]:
        T, Dp = ck["T"], ck["Dp"]
        lamL = hotrg.eigh_desc(hotrg.gram(T))[0]
        lamR = hotrg.eigh_desc(hotrg.gram(hotrg.swap_lr(T)))[0]
        assert abs(np.sum(lamL) - np.sum(lamR)) < 1e-12 * np.sum(lamL)   # same trace
        eL, eR = np.sum(lamL[Dp:]), np.sum(lamR[Dp:])
        want = 1 if eL - eR > hotrg.W_RULE_TIE * np.sum(lamL) else 0
        assert ck["side"] == want
        assert abs(np.sum(ck["lam"][Dp:]) - (eR if want else eL)) <= 1e-15 * np.sum(lamL)
        sides.append(ck["side"])
    assert 1 in sides and 0 in sides          # the rule actually switches on this input


def test_w_rule_1_gradient_against_finite_differences_and_euler_identity():
    import synth
    T0 = synth.random_T0(3, 3)
    D, n = 5, 4
    fwd = hotrg.hotrg_forward(T0, D, n, w_rule=1)
    g = hotrg.hotrg_backward(fwd)
    f = lambda T: hotrg.hotrg_forward(T, D, n, keep=False, w_rule=1)["lnz"]
    rng = np.random.default_rng(0)
    for flat in rng.choice(T0.size, 10, replace=False):
        idx = np.unravel_index(flat, T0.shape)
        Tp, Tm = T0.copy(), T0.copy()
        Tp[idx] += 1e-6
        Tm[idx] -= 1e-6
        fd = (f(Tp) - f(Tm)) / 2e-6
        assert abs(fd - g[idx]) < 1e-7 * np.abs(g).max()
    assert abs(float(np.sum(T0 * g)) - 1.0) < 1e-10
    assert any(ck["side"] == 1 for ck in fwd["ckpt"])
