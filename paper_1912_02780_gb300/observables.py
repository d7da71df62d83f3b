"""Thermodynamics of the square-lattice Ising model from HOTRG solves.

For each inverse temperature beta on a grid the library returns ln Z / N and,
from the hand-written backward, d(ln Z / N)/d beta.  From these:

    f(beta) = -ln Z / (N beta)                      free energy per site
    u(beta) = -d(ln Z / N)/d beta                    internal energy per site
    c(beta) = beta^2 d^2(ln Z / N)/d beta^2 = -beta^2 du/dbeta

The paper obtains such derivatives numerically (main text, energy as the
derivative of beta f); here u comes from the adjoint and c from a
second-order finite difference of u on the grid (central inside, one-sided
at the two ends), the same rule the oracle applies to its own u.
"""
from __future__ import annotations

import numpy as np

from . import Plan


def grid_derivative(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Second-order finite-difference dy/dx on a uniform grid (central inside,
    one-sided three-point at the ends)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    h = x[1] - x[0]
    d = np.empty_like(y)
    d[1:-1] = (y[2:] - y[:-2]) / (2 * h)
    d[0] = (-3 * y[0] + 4 * y[1] - y[2]) / (2 * h)
    d[-1] = (3 * y[-1] - 4 * y[-2] + y[-3]) / (2 * h)
    return d


def ising_thermodynamics(betas, d_cut: int, n_steps: int, precision: str = "fp64",
                         split_from_step: int = 1, J: float = 1.0, h: float = 0.0,
                         hi_precision_steps: int = 2, concurrent: int = 1,
                         sm_reserve: int = 0, grouped: int = 0) -> dict:
    """ln Z / N, f, u and c on a beta grid.  ``concurrent`` plans, each on its
    own CUDA stream and host thread, take the betas round-robin (so that one
    solve's latency-bound eigensolver kernels run beside another's
    contractions; ``sm_reserve`` SMs are left free by each plan's
    contraction GEMMs for that).  ``grouped`` > 1 (split precision): the betas
    go in batches of that many through one grouped forward each (every
    contraction stage of the batch one tensor-core launch), then each plan's
    backward.  Every beta's result is the same as with one plan."""
    import threading
    betas = np.asarray(betas, dtype=np.float64)
    lnz = np.empty_like(betas)
    dlnz = np.empty_like(betas)
    if grouped > 1 and precision != "fp64":
        import torch
        from . import Group
        G = min(int(grouped), len(betas))
        st = torch.cuda.Stream()
        kw = dict(split_from_step=split_from_step, want_grad=True,
                  hi_precision_steps=hi_precision_steps)
        plans = [Plan(2, d_cut, n_steps, precision, stream=st.cuda_stream, **kw)
                 for _ in range(G)]
        try:
            with Group(2, d_cut, n_steps, precision, max_count=G, stream=st.cuda_stream,
                       **kw) as grp:
                for i0 in range(0, len(betas), G):
                    bs = betas[i0:i0 + G]
                    ps = plans[:len(bs)]
                    lnz[i0:i0 + len(bs)] = grp.forward_ising(ps, bs, J, h)
                    for j, p in enumerate(ps):
                        _, dlnz[i0 + j] = p.backward(want_dbeta=True)
        finally:
            for p in plans:
                p.close()
        u = -dlnz
        c = (-betas ** 2 * grid_derivative(betas, u) if len(betas) >= 3
             else np.full_like(betas, np.nan))
        return dict(beta=betas, lnz=lnz, f=-lnz / betas, u=u, c=c)
    C = max(1, min(int(concurrent), len(betas)))
    streams = []
    if C > 1:
        import torch
        streams = [torch.cuda.Stream() for _ in range(C)]
    plans = [Plan(2, d_cut, n_steps, precision, split_from_step=split_from_step, want_grad=True,
                  hi_precision_steps=hi_precision_steps,
                  stream=streams[c].cuda_stream if streams else None,
                  gemm_sm_reserve=sm_reserve if C > 1 else 0) for c in range(C)]
    errors = []

    def run(c):
        try:
            for i in range(c, len(betas), C):
                lnz[i], _, _ = plans[c].forward_ising(float(betas[i]), J, h)
                _, dlnz[i] = plans[c].backward(want_dbeta=True)
        except Exception as e:          # re-raised in the caller's thread
            errors.append(e)

    try:
        if C == 1:
            run(0)
        else:
            threads = [threading.Thread(target=run, args=(c,)) for c in range(C)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
    finally:
        for p in plans:
            p.close()
    if errors:
        raise errors[0]
    u = -dlnz
    c = -betas ** 2 * grid_derivative(betas, u) if len(betas) >= 3 else np.full_like(betas, np.nan)
    return dict(beta=betas, lnz=lnz, f=-lnz / betas, u=u, c=c)
