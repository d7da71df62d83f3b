"""w_rule = 1 (the isometry from whichever of the left and right Gram
matrices discards less, Xie2012's rule) on the GPU against the oracle:
forward, the side of every step, and the gradient through the chosen side."""
import numpy as np
import pytest

import synth
from oracle import hotrg, ising

pytestmark = pytest.mark.gpu
hot = pytest.importorskip("paper_1912_02780_gb300")


def _margins(fwd):
    """Relative differences of the left and right discarded weights per step."""
    out = []
    for ck in fwd["ckpt"]:
        T, Dp = ck["T"], ck["Dp"]
        lamL = hotrg.eigh_desc(hotrg.gram(T))[0]
        lamR = hotrg.eigh_desc(hotrg.gram(hotrg.swap_lr(T)))[0]
        out.append((np.sum(lamL[Dp:]) - np.sum(lamR[Dp:])) / np.sum(lamL))
    return out


def test_forward_and_sides_against_oracle():
    T0 = synth.random_T0(3, 3)
    D, n = 5, 6
    ref = hotrg.hotrg_forward(T0, D, n, w_rule=1)
    assert min(abs(m) for m in _margins(ref)) > 1e-3        # no near-ties on this input
    with hot.Plan(3, D, n, want_grad=False, w_rule=1) as p:
        lnz, ln, _ = p.forward_tensor(T0)
        sides = p.isometry_sides()
    assert list(sides) == [ck["side"] for ck in ref["ckpt"]]
    assert 1 in sides
    assert abs(lnz - ref["lnz"]) < 1e-12
    assert np.abs(ln - np.array(ref["log_norms"])).max() < 1e-12


def test_gradient_through_the_chosen_side_against_oracle():
    T0 = synth.random_T0(3, 3)
    D, n = 5, 4
    fwd = hotrg.hotrg_forward(T0, D, n, w_rule=1)
    g_ref = hotrg.hotrg_backward(fwd)
    with hot.Plan(3, D, n, want_grad=True, w_rule=1) as p:
        p.forward_tensor(T0)
        g = p.backward()
    assert np.abs(g - g_ref).max() / np.abs(g_ref).max() < 1e-9
    assert abs(float(np.sum(T0 * g)) - 1.0) < 1e-10


def test_symmetric_tensor_takes_the_left_side_bit_for_bit():
    T0 = ising.ising_T0(0.44, 1.0, 0.0)
    with hot.Plan(2, 8, 12, want_grad=True) as p:
        a = p.forward_tensor(T0)[0]
        ga = p.backward()
    with hot.Plan(2, 8, 12, want_grad=True, w_rule=1) as p:
        b = p.forward_tensor(T0)[0]
        gb = p.backward()
        assert not p.isometry_sides().any()
    assert a == b and np.array_equal(ga, gb)


def test_split_precision_follows_fp64():
    T0 = synth.random_T0(5, 4)
    D, n = 16, 8
    with hot.Plan(4, D, n, "fp64", want_grad=False, w_rule=1) as p:
        ref = p.forward_tensor(T0)[0]
        s_ref = p.isometry_sides()
    with hot.Plan(4, D, n, "bf16x6", split_from_step=3, want_grad=False, w_rule=1) as p:
        got = p.forward_tensor(T0)[0]
        s_got = p.isometry_sides()
    assert np.array_equal(s_ref, s_got)
    assert abs(got - ref) < 1e-9


def test_w_rule_rejected_with_given_isometries():
    with pytest.raises(hot.HotrgError):
        hot.Plan(2, 8, 4, want_grad=True, fixed_w_grad=True, w_given=True, w_rule=1)
