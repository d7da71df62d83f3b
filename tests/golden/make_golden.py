"""Write stored expected values for the GPU parity tests and the benchmark.

Calls only the FP64 oracle (oracle/) and the seeded input generators
(synth/); nothing here touches the CUDA path.  Each case writes
tests/golden/<name>.json with the oracle's ln Z / N, per-step log-norms and,
where requested, d(ln Z/N)/d T0 and d(ln Z/N)/d beta.

Usage: python tests/golden/make_golden.py <case> [<case> ...]
Cases:
  c4_d64_s0   random reflection-symmetric T0 (d0 = 4, seed 0), D_cut = 64, 30 steps (forward)
  c4_d64_s1   same, seed 1
  c3_bc_h0    Ising at beta_c, h = 0, D_cut = 64, 40 steps (forward)
  c3_bc_h001  Ising at beta_c, h = 0.01, D_cut = 64, 40 steps (forward)
  c3_bc_h0_grad, c3_bc_h001_grad
              the same two Ising cases with the full backward: d(ln Z/N)/d T0 (16
              entries, per site, w(T) differentiated) and d(ln Z/N)/d beta
  c1_ising    Ising at beta = 0.44, h = 0, D_cut = 8, 20 steps (forward + full backward)
  c2_grid     Ising, 64 betas on [0.30, 0.60], D_cut = 32, 30 steps (forward + d/dbeta)
  c4_d96_s0_n7  random T0 (d0 = 4, seed 0), D_cut = 96, 7 steps (forward; steps 5-7 at the
              full D_cut = 96 bond dimensions)
  c4_d96_s0   the same tensor, D_cut = 96, 30 steps (forward; hours on the CPU)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import hotrg, ising  # noqa: E402
import synth  # noqa: E402


def fwd_case(name, T0, d_cut, n, meta):
    t = time.time()
    f = hotrg.hotrg_forward(T0, d_cut, n, keep=False)
    out = dict(meta, d_cut=d_cut, n_steps=n, lnz=f["lnz"], log_norms=f["log_norms"],
               trace_sign=f["trace_sign"], trunc_err=f["trunc_err"],
               cut_gap=[g if np.isfinite(g) else None for g in f["cut_gap"]],
               oracle_seconds=time.time() - t)
    json.dump(out, open(os.path.join(HERE, name + ".json"), "w"), indent=1)
    print(name, out["lnz"], f"{out['oracle_seconds']:.1f}s", flush=True)


def grad_case(name, beta, J, h, d_cut, n):
    """Forward with checkpoints, then the oracle's reverse-mode backward
    (SM Sec. B recursion, SM Sec. E chain rule, eigensolve adjoint)."""
    t = time.time()
    T0 = ising.ising_T0(beta, J, h)
    f = hotrg.hotrg_forward(T0, d_cut, n, keep=True)
    t_fwd = time.time() - t
    g = hotrg.hotrg_backward(f)
    db = float(np.sum(g * ising.ising_dT0_dbeta(beta, J, h)))
    out = dict(model="ising", beta=beta, J=J, h=h, d0=2, d_cut=d_cut, n_steps=n,
               lnz=f["lnz"], log_norms=f["log_norms"], trace_sign=f["trace_sign"],
               trunc_err=f["trunc_err"],
               cut_gap=[x if np.isfinite(x) else None for x in f["cut_gap"]],
               dlnz_dT0=[float(v) for v in g.ravel()], dlnz_dbeta=db,
               euler=float(np.sum(g * T0)), eta_rel=hotrg.ETA_REL_DEFAULT,
               oracle_seconds_forward=t_fwd, oracle_seconds=time.time() - t)
    json.dump(out, open(os.path.join(HERE, name + ".json"), "w"), indent=1)
    print(name, out["lnz"], db, out["euler"], f"{out['oracle_seconds']:.1f}s", flush=True)


def main(cases):
    for c in cases:
        if c.startswith("c4_d64_s"):
            seed = int(c[len("c4_d64_s"):])
            fwd_case(c, synth.random_symmetric_T0(seed, 4), 64, 30,
                     dict(model="random reflection-symmetric T0", d0=4, seed=seed))
        elif c == "c4_d96_s0":
            fwd_case(c, synth.random_symmetric_T0(0, 4), 96, 30,
                     dict(model="random reflection-symmetric T0", d0=4, seed=0))
        elif c == "c4_d96_s0_n7":
            fwd_case(c, synth.random_symmetric_T0(0, 4), 96, 7,
                     dict(model="random reflection-symmetric T0", d0=4, seed=0))
        elif c == "c3_bc_h0":
            fwd_case(c, ising.ising_T0(synth.BETA_C, 1.0, 0.0), 64, 40,
                     dict(model="ising", beta=synth.BETA_C, J=1.0, h=0.0, d0=2))
        elif c == "c3_bc_h001":
            fwd_case(c, ising.ising_T0(synth.BETA_C, 1.0, 0.01), 64, 40,
                     dict(model="ising", beta=synth.BETA_C, J=1.0, h=0.01, d0=2))
        elif c == "c1_ising":
            grad_case(c, 0.44, 1.0, 0.0, 8, 20)
        elif c == "c3_bc_h0_grad":
            grad_case(c, synth.BETA_C, 1.0, 0.0, 64, 40)
        elif c == "c3_bc_h001_grad":
            grad_case(c, synth.BETA_C, 1.0, 0.01, 64, 40)
        elif c == "c2_grid":
            res = []
            t = time.time()
            for b in synth.beta_grid():
                f = hotrg.hotrg_forward(ising.ising_T0(b), 32, 30)
                g = hotrg.hotrg_backward(f)
                db = float(np.sum(g * ising.ising_dT0_dbeta(b)))
                res.append(dict(beta=float(b), lnz=f["lnz"], dlnz_dbeta=db))
                print(f"beta={b:.4f} lnz={f['lnz']:.15f} dbeta={db:.12f}", flush=True)
            json.dump(dict(model="ising", J=1.0, h=0.0, d0=2, d_cut=32, n_steps=30, points=res,
                           oracle_seconds=time.time() - t),
                      open(os.path.join(HERE, c + ".json"), "w"), indent=1)
        else:
            raise SystemExit(f"unknown case {c}")


if __name__ == "__main__":
    main(sys.argv[1:])
