"""Failure detection without a GPU fault: bounded device waits report a
timeout status, host-injected failures surface as the documented status
codes, invalid calls are rejected, and a plan stays usable after any error."""
import math
import time

import numpy as np
import pytest

import synth
from oracle import hotrg, ising

pytestmark = pytest.mark.gpu
hot = pytest.importorskip("paper_1912_02780_gb300")


@pytest.fixture(autouse=True)
def _reset_injection():
    yield
    hot.lib().hotrg_debug_inject(0, 0)


def test_bounded_wait_gives_up_and_reports_timeout():
    L = hot.lib()
    t0 = time.time()
    assert L.hotrg_check_bounded_wait(20.0) == 6          # HOTRG_ETIMEOUT
    assert time.time() - t0 < 10.0
    # the context is still usable afterwards
    rng = np.random.default_rng(0)
    A, B = rng.standard_normal((64, 64)), rng.standard_normal((32, 64))
    assert np.allclose(hot.gemm_f64_check(A, B), A @ B.T, atol=1e-12)


def test_injected_allocation_failure_then_recovery():
    L = hot.lib()
    L.hotrg_debug_inject(1, 3)
    with pytest.raises(hot.HotrgError) as ei:
        hot.Plan(2, 8, 10, "fp64")
    assert ei.value.status == 2                          # HOTRG_ENOMEM
    L.hotrg_debug_inject(0, 0)
    with hot.Plan(2, 8, 10, "fp64", want_grad=False) as p:
        lnz, _, _ = p.forward_ising(0.44)
    assert abs(lnz - hotrg.hotrg_forward(ising.ising_T0(0.44), 8, 10, keep=False)["lnz"]) < 1e-12


@pytest.mark.parametrize("what,status", [(2, 4), (3, 5)])   # ENOTCONV, ENONFINITE
def test_injected_device_failures_and_plan_reuse(what, status):
    L = hot.lib()
    ref = hotrg.hotrg_forward(ising.ising_T0(0.44), 8, 12, keep=False)["lnz"]
    with hot.Plan(2, 8, 12, "fp64") as p:
        L.hotrg_debug_inject(what, 4)
        with pytest.raises(hot.HotrgError) as ei:
            p.forward_ising(0.44)
        assert ei.value.status == status
        # backward after a failed forward is refused
        with pytest.raises(hot.HotrgError) as eb:
            p.backward()
        assert eb.value.status == 7                      # HOTRG_ESTATE
        L.hotrg_debug_inject(0, 0)
        lnz, _, _ = p.forward_ising(0.44)
        assert abs(lnz - ref) < 1e-12
        p.backward()


def test_invalid_calls_are_rejected():
    with pytest.raises(hot.HotrgError) as e1:
        hot.Plan(2, 0, 10)
    assert e1.value.status == 1
    with hot.Plan(2, 8, 6, "fp64") as p:
        with pytest.raises(hot.HotrgError) as e2:
            p.backward()                                  # no forward yet
        assert e2.value.status == 7
        bad = ising.ising_T0(0.4)
        bad[0, 0, 0, 0] = math.nan
        with pytest.raises(hot.HotrgError) as e3:
            p.forward_tensor(bad)
        assert e3.value.status == 1
        with pytest.raises(hot.HotrgError) as e4:
            p.forward_ising(0.4, -1.0, 0.0)               # beta J < 0
        assert e4.value.status == 1
    with hot.Plan(4, 8, 6, "fp64") as p4:
        with pytest.raises(hot.HotrgError):
            p4.forward_ising(0.4)                         # Ising needs d0 = 2
    with hot.Plan(2, 8, 6, "fp64", want_grad=False) as p:
        p.forward_ising(0.4)
        with pytest.raises(hot.HotrgError) as e5:
            p.backward()                                  # plan without gradients
        assert e5.value.status == 7
