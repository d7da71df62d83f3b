"""Solve server: results are the same alone and in the concurrent mix, the
device-memory budget is respected, oversized requests are rejected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

hot = pytest.importorskip("paper_1912_02780_gb300")

MIX = [  # (beta, h, d_cut, n_steps, want_grad, precision, split_from)
    (0.30, 0.00, 8, 12, True, "fp64", 1),
    (0.44, 0.01, 16, 14, False, "fp64", 1),
    (0.50, 0.02, 16, 10, True, "bf16x6", 5),
    (0.35, 0.00, 8, 16, False, "fp64", 1),
    (0.60, 0.05, 16, 12, True, "fp64", 1),
    (0.41, 0.03, 16, 14, True, "bf16x6", 5),
    (0.47, 0.00, 8, 10, True, "fp64", 1),
    (0.33, 0.04, 16, 16, False, "bf16x6", 5),
    (0.55, 0.01, 8, 14, False, "fp64", 1),
    (0.44, 0.00, 16, 12, True, "fp64", 1),
]


def alone(beta, h, d_cut, n, grad, prec, sf):
    # the server's configuration of a request: forward-only requests use the
    # randomized subspace eigensolver with two power iterations, warm-started
    # from step k - 2 (the SMs the server's plans leave free do not change
    # any result)
    with hot.Plan(2, d_cut, n, prec, split_from_step=sf, want_grad=grad,
                  eigh_mode=0 if grad else 1, eigh_power_iters=2,
                  eigh_warm_start=0 if grad else 1) as p:
        lnz, _, _ = p.forward_ising(beta, 1.0, h)
        db = p.backward(want_dbeta=True)[1] if grad else 0.0
    return lnz, db


def test_results_same_alone_and_in_mix():
    ref = [alone(*m) for m in MIX]
    with hot.Server(hbm_budget_bytes=40 << 30, max_slots=3) as srv:
        tickets = [srv.submit(b, 1.0, h, d, n, g, pr, sf) for (b, h, d, n, g, pr, sf) in MIX]
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(MIX) and st["failed"] == 0
    slots = set()
    for (lnz, db), r, m in zip(ref, res, MIX):
        assert r.status == 0
        slots.add(r.slot)
        assert abs(r.lnz_per_site - lnz) < 1e-12
        if m[4]:
            assert abs(r.dlnz_dbeta - db) < 1e-10 * max(1.0, abs(db))
        assert r.t_submit <= r.t_start <= r.t_finish
    assert len(slots) > 1        # the mix really ran on several slots


def test_budget_admission_and_rejection():
    b16 = hot.workspace_bytes(2, 16, 14, want_grad=True)
    with hot.Server(hbm_budget_bytes=int(1.5 * b16), max_slots=3) as srv:
        ts = [srv.submit(0.44, 1.0, 0.0, 16, 14, True) for _ in range(4)]
        big = srv.submit(0.44, 1.0, 0.0, 64, 30, True)          # plan far beyond the budget
        res = [srv.wait(t) for t in ts]
        rb = srv.wait(big)
        st = srv.stats()
    assert all(r.status == 0 for r in res)
    assert rb.status == 2                                       # HOTRG_ENOMEM
    assert st["peak_bytes"] <= int(1.5 * b16)
    lnz = [r.lnz_per_site for r in res]
    assert max(lnz) - min(lnz) < 1e-13


def test_same_shape_requests_run_as_a_grouped_forward():
    """Forward-only split requests of one D_cut queued together run as one
    grouped forward (their contractions one tensor-core launch per stage);
    every result equals the request's own solve bit for bit."""
    reqs = [(0.30 + 0.05 * i, 0.01 * i, 16, 12 + (i % 3), False, "bf16x6", 5) for i in range(6)]
    ref = [alone(*m) for m in reqs]
    with hot.Server(hbm_budget_bytes=40 << 30, max_slots=1) as srv:
        tickets = [srv.submit(b, 1.0, h, d, n, g, pr, sf) for (b, h, d, n, g, pr, sf) in reqs]
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["failed"] == 0 and st["grouped"] >= 2 and st["groups"] >= 1
    for (lnz, _), r in zip(ref, res):
        assert r.status == 0
        assert r.lnz_per_site == lnz
