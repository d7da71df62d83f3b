"""The C-ABI library builds, loads without a GPU and exports every symbol
declared in include/hotrg.h; host-side logic (config defaults, workspace
sizing, argument validation) works on the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hotrg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hotrg_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def hot():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_02780_gb300 as hot
    return hot


def test_exports_every_declared_symbol(hot):
    L = hot.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hot.EXPORTS)


def test_config_defaults(hot):
    c = hot.make_config(2, 8, 20)
    assert (c.d0, c.d_cut, c.n_steps, c.precision, c.split_from_step) == (2, 8, 20, 0, 1)
    assert c.want_grad == 1 and c.fixed_w_grad == 0 and c.eigh_broadening == 1e-12


def test_workspace_bytes_grows_with_d_cut(hot):
    a = hot.workspace_bytes(2, 16, 20)
    b = hot.workspace_bytes(2, 32, 20)
    c = hot.workspace_bytes(4, 64, 30, precision="bf16x3")
    assert 0 < a < b < c
    # D = 64, 30 steps with gradients: checkpoints + eigenvectors dominate, tens of GB at most
    assert c < 80 * 2 ** 30


def test_invalid_configs_rejected(hot):
    L = hot.lib()
    for args in [(0, 8, 4), (2, 0, 4), (2, 8, 0)]:
        c = hot.make_config(*args)
        out = ctypes.c_size_t(0)
        assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1
    c = hot.make_config(2, 8, 4)
    c.precision = 7
    out = ctypes.c_size_t(0)
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1


def test_status_strings(hot):
    L = hot.lib()
    assert L.hotrg_status_string(0) == b"ok"
    assert L.hotrg_status_string(6) == b"device wait timed out"


def test_split_chunk_budget_shrinks_the_plan(hot):
    kw = dict(precision="bf16x6", split_from_step=4, want_grad=False, hi_precision_steps=3,
              eigh_mode=1, eigh_power_iters=2)
    full = hot.workspace_bytes(4, 64, 7, **kw)
    small = hot.workspace_bytes(4, 64, 7, split_chunk_elems=1 << 26, **kw)
    assert small < full / 4          # the y-chunked D^5 stage buffers dominate at D_cut = 64
    L = hot.lib()
    c = hot.make_config(4, 64, 7, split_chunk_elems=-1, **kw)
    out = ctypes.c_size_t(0)
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1


def test_w_given_needs_fixed_w_gradients(hot):
    L = hot.lib()
    out = ctypes.c_size_t(0)
    c = hot.make_config(2, 8, 6, w_given=True)                 # fixed_w_grad = 0
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1
    c = hot.make_config(2, 8, 6, w_given=True, fixed_w_grad=True, want_grad=False)
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1
    c = hot.make_config(2, 8, 6, w_given=True, fixed_w_grad=True)
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 0


def test_dtrg_driver_needs_one_input():
    from paper_1912_02780_gb300.dtrg import dtrg_sweeps
    with pytest.raises(ValueError):
        dtrg_sweeps(2, 6, 4, n_sweeps=1)                                  # neither T0 nor beta
    with pytest.raises(ValueError):
        dtrg_sweeps(2, 6, 4, n_sweeps=1, T0=np.ones((2, 2, 2, 2)), beta=0.4)   # both


def test_scheme_w_rule_and_group_host_checks(hot):
    """Host-side validation and sizing of the scheme-(b), w_rule and grouped
    forward options (no GPU needed)."""
    L = hot.lib()
    out = ctypes.c_size_t(0)
    bad = [dict(scheme=2), dict(scheme=-1), dict(w_rule=2),
           dict(w_rule=1, want_grad=True, fixed_w_grad=True, w_given=True)]
    for kw in bad:
        c = hot.make_config(4, 16, 8, **kw)
        assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1, kw
    c = hot.make_config(4, 16, 8, scheme=1)
    c.chain_steps = 2                      # the binding passes 0 / 1; the library checks
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1
    c = hot.make_config(4, 5000, 8, scheme=1)
    assert L.hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 1
    # scheme (b) keeps the vertical legs at d0: much smaller than scheme (a) at the same D_cut
    a = hot.workspace_bytes(4, 64, 12, want_grad=False)
    b = hot.workspace_bytes(4, 64, 12, want_grad=False, scheme=1)
    assert 0 < b < a
    # w_rule 1 adds the right side's eigenvectors
    assert hot.workspace_bytes(4, 16, 8, w_rule=1) > hot.workspace_bytes(4, 16, 8)
    # grouped-forward buffers: none without split steps, growing with the group size
    def gbytes(cfg, count):
        n = ctypes.c_size_t(0)
        assert L.hotrg_group_workspace_bytes(ctypes.byref(cfg), count, ctypes.byref(n)) == 0
        return n.value
    assert gbytes(hot.make_config(2, 16, 20), 4) == 0
    cs = hot.make_config(2, 16, 20, precision="bf16x6", split_from_step=5)
    assert 0 < gbytes(cs, 2) < gbytes(cs, 4)
    n = ctypes.c_size_t(0)
    assert L.hotrg_group_workspace_bytes(ctypes.byref(cs), 0, ctypes.byref(n)) == 1
    assert L.hotrg_group_workspace_bytes(ctypes.byref(cs), 65, ctypes.byref(n)) == 1


def test_xy_per_site_conversion_matches_oracle():
    """The scheme-(b) driver's conversion of ln Z per copy of T0 to per-site
    thermodynamics agrees with the oracle's."""
    from oracle import xtrg
    from paper_1912_02780_gb300 import xtrg as gx
    out = np.array([0.7, 0.35, 0.18])
    depths = np.array([1, 2, 3])
    tau = 0.01
    beta, lnz_site, f = gx.per_site(out, depths, tau)
    for k, o, b, l, ff in zip(depths, out, beta, lnz_site, f):
        assert b == tau * 2.0 ** (k + 1)
        assert abs(l - xtrg.lnz_per_site(o, k + 1)) < 1e-15
        assert abs(ff + l / b) < 1e-15
