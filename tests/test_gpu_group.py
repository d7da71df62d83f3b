"""Grouped forward: several plans of one shape stepped in lockstep, the
contractions of all of them one tensor-core launch per stage.  Every result
must equal the plan's own forward bit for bit (the same kernels do the same
arithmetic per problem), at any mix of depths, and a backward after a grouped
forward must equal the one after the plan's own forward."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
hot = pytest.importorskip("paper_1912_02780_gb300")
torch = pytest.importorskip("torch")


def _stream():
    return torch.cuda.Stream(torch.device("cuda", 0))


@pytest.mark.parametrize("d_cut,split_from", [(16, 5), (24, 5)])
def test_grouped_ising_equals_each_plans_own_forward(d_cut, split_from):
    kw = dict(split_from_step=split_from, want_grad=False, hi_precision_steps=2)
    betas = [0.30, 0.40, 0.4406867935097715, 0.50, 0.60]
    n = 20
    st = _stream()
    plans = [hot.Plan(2, d_cut, n, "bf16x6", stream=st.cuda_stream, **kw) for _ in betas]
    try:
        ref = [p.forward_ising(b)[0] for p, b in zip(plans, betas)]
        ref_ln = []
        for p, b in zip(plans, betas):
            ref_ln.append(p.forward_ising(b)[1])
        with hot.Group(2, d_cut, n, "bf16x6", max_count=8, stream=st.cuda_stream, **kw) as g:
            l0 = hot.kernel_launches()
            got = g.forward_ising(plans, betas)
            grouped_calls = hot.kernel_launches() - l0
            assert g.launches() > 0
        for i, p in enumerate(plans):
            assert got[i] == ref[i]
            # the plan's own outputs after the grouped forward
            lnz, ln, _ = p.forward_ising(betas[i])
            assert lnz == ref[i] and np.array_equal(ln, ref_ln[i])
        l0 = hot.kernel_launches()
        for p, b in zip(plans, betas):
            p.forward_ising(b)
        single_calls = hot.kernel_launches() - l0
        assert grouped_calls < single_calls
    finally:
        for p in plans:
            p.close()


def test_grouped_mixed_depths_and_tensors():
    kw = dict(split_from_step=4, want_grad=False, hi_precision_steps=3)
    D, n = 16, 12
    depths = [12, 9, 7, 12]
    T0s = [synth.random_symmetric_T0(s, 4) for s in range(len(depths))]
    st = _stream()
    plans = [hot.Plan(4, D, n, "bf16x6", stream=st.cuda_stream, **kw) for _ in depths]
    try:
        ref = []
        for p, d, T0 in zip(plans, depths, T0s):
            p.set_steps(d)
            ref.append(p.forward_tensor(T0)[0])
        with hot.Group(4, D, n, "bf16x6", max_count=4, stream=st.cuda_stream, **kw) as g:
            got = g.forward_tensor(plans, np.stack(T0s))
        assert list(got) == ref
    finally:
        for p in plans:
            p.close()


def test_backward_after_grouped_forward():
    kw = dict(split_from_step=5, want_grad=True, hi_precision_steps=2)
    D, n = 16, 12
    betas = [0.42, 0.46]
    st = _stream()
    plans = [hot.Plan(2, D, n, "bf16x6", stream=st.cuda_stream, **kw) for _ in betas]
    try:
        ref = []
        for p, b in zip(plans, betas):
            p.forward_ising(b)
            ref.append(p.backward(want_dbeta=True))
        with hot.Group(2, D, n, "bf16x6", max_count=2, stream=st.cuda_stream, **kw) as g:
            g.forward_ising(plans, betas)
        for p, (g0, db0) in zip(plans, ref):
            g1, db1 = p.backward(want_dbeta=True)
            assert np.array_equal(g1, g0) and db1 == db0
    finally:
        for p in plans:
            p.close()


def test_group_rejects_other_shapes():
    st = _stream()
    kw = dict(split_from_step=5, want_grad=False)
    with hot.Group(2, 16, 12, "bf16x6", max_count=2, stream=st.cuda_stream, **kw) as g:
        a = hot.Plan(2, 16, 12, "bf16x6", stream=st.cuda_stream, **kw)
        b = hot.Plan(2, 24, 12, "bf16x6", stream=st.cuda_stream, **kw)
        try:
            for bad in ([a, b], [a, a], [a, a, a]):
                with pytest.raises(hot.HotrgError):
                    g.forward_ising(bad, 0.4)
        finally:
            for p in (a, b):
                p.close()


def test_grouped_plans_on_their_own_streams():
    """Plans on streams of their own (their eigensolves overlap), the grouped
    contractions on the group's stream: the same results, bit for bit, over
    repeated calls (every ordering between the streams comes from events)."""
    kw = dict(split_from_step=5, want_grad=False, hi_precision_steps=2, eigh_mode=1,
              eigh_power_iters=2, eigh_warm_start=1)
    betas = [0.36, 0.41, 0.44, 0.52]
    streams = [_stream() for _ in betas]
    gs = _stream()
    plans = [hot.Plan(2, 16, 24, "bf16x6", stream=st.cuda_stream, **kw) for st in streams]
    try:
        ref = [p.forward_ising(b)[0] for p, b in zip(plans, betas)]
        with hot.Group(2, 16, 24, "bf16x6", max_count=4, stream=gs.cuda_stream, **kw) as g:
            for _ in range(3):
                got = g.forward_ising(plans, betas)
                assert list(got) == ref
    finally:
        for p in plans:
            p.close()
