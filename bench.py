"""Benchmark of the HOTRG hot path on GB300.

Workload (default): the split-precision configuration of the headline metric,
seeded random reflection-symmetric rank-4 tensors T0 (bond dimension 4,
entries N(0,1), max|T| = 1; seeds 0-4), D_cut = 64, 30 coarse-graining steps,
the O(D^7) contractions and the Gram matrices on the tensor cores in split
BF16 (four planes on the first --hi-steps split steps, three after; exact
hi*hi accumulation), the eigensolve (randomized subspace iteration with
Rayleigh-Ritz, or cuSOLVER's partial solver), norms and log-norm accumulation
in FP64;
steps before --split-from run entirely in FP64.  One benchmark step = the
solves of the --concurrent seeds (default 2: seeds 0 and 1), each on its own stream
and host thread (forward; with --grad also the backward).

Printed: one JSON line (rank 0) with solves/s over all GPUs, useful and
executed TFLOP/s, the roofline of the dominant kernel (stage-2 tensor-core
GEMM) measured with CUDA events on the plan's stream, SM clocks sampled during
the timed region, an end-to-end number through the host-buffer C ABI, the
FP64 CPU oracle timed on a bounded sample of the same workload, and the error
of this run against the oracle's stored result when one exists.

--impl reference times the FP64 CPU oracle itself (the reference arm) on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    # name: (d0, d_cut, n_steps, description)
    "c4_d64": (4, 64, 30, "random reflection-symmetric T0 d0=4 seed 0, D_cut=64, 30 steps"),
    "c4_d96": (4, 96, 30, "random reflection-symmetric T0 d0=4 seed 0, D_cut=96, 30 steps"),
    "c4_d32": (4, 32, 30, "random reflection-symmetric T0 d0=4 seed 0, D_cut=32, 30 steps"),
}


def schedule(d0, d_cut, n):
    """Per-step (X, Y, X') of the bond-dimension schedule."""
    out = []
    X = Y = d0
    for _ in range(n):
        Xp = min(X * X, d_cut)
        out.append((X, Y, Xp))
        X, Y = Y, Xp
    return out


def step_flops(X, Y, Xp):
    """Useful forward flops of one step (one MAC = 2 flops): Gram halves A, B
    (2 X^3 Y^3 each), G (2 X^4 Y^2), stage 1 (2 X^3 Y^2 X'), stage 2
    (2 X^3 Y^3 X'), stage 3 (2 X^2 Y^2 X'^2)."""
    gram = 4 * X ** 3 * Y ** 3 + 2 * X ** 4 * Y ** 2
    s1 = 2 * X ** 3 * Y ** 2 * Xp
    s2 = 2 * X ** 3 * Y ** 3 * Xp
    s3 = 2 * X ** 2 * Y ** 2 * Xp ** 2
    return dict(gram=gram, s1=s1, s2=s2, s3=s3, total=gram + s1 + s2 + s3)


def is_split_step(k, X, Y, Xp, split_from, precision):
    return precision != "fp64" and k >= split_from and X % 8 == 0 and Y % 8 == 0 and Xp % 8 == 0


def products_of_step(k, split_from, hi_steps, precision):
    """Tensor-core products per K step of a split step (BF16X6: four planes /
    10 products on the first hi_steps split steps, three planes / 6 after)."""
    if precision == "bf16x3":
        return 3
    return 10 if k < split_from + hi_steps else 6


# DRAM traffic of one stage-2 launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the tensor-core GEMM source with this SHA-256; the
# value is reported only while csrc/gemm_tc.cu is unchanged since the capture.
STAGE2_TRAFFIC = {
    "gemm_tc_sha256": "e71848dcbe2214a6f30c74c75d170e62260694ed98df8242db7fe1e3aa06a245",
    # full-size D = 64 three-plane stage-2 launch (step 7 of the benchmark's
    # solve: N-tile groups of 16, 136 CTAs with 16 SMs reserved, 44.46 ms under
    # ncu), one-pass ncu capture: 48.25 GB read + 8.67 GB written
    "bytes_per_launch_d64": 48.25e9 + 8.67e9,
    "captured": "profiles/tc_gemm_stage2_c4_d64.md"}


def gemm_source_sha():
    import hashlib
    path = os.path.join(ROOT, "paper_1912_02780_gb300", "csrc", "gemm_tc.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def aggregate_over_ranks(ms_local, solves_local, dist=None, device=None):
    """Whole-job throughput: the max elapsed time over ranks and the sum of
    solves over ranks (independent replicas).  Returns (ms_max, solves_total)."""
    if dist is None:
        return ms_local, solves_local
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(solves_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def golden(name):
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", name + ".json")))
    except (OSError, ValueError):
        return None


def oracle_sample(d_cut, seconds_cap=60.0):
    """Time the FP64 CPU oracle on one steady coarse-graining step of the
    workload (X = Y = X' = d_cut): Gram, eigensolve, contraction, norm.
    Returns (seconds, flops of that step)."""
    from oracle import hotrg
    rng = np.random.default_rng(0)
    D = d_cut
    T = rng.standard_normal((D, D, D, D))
    T /= np.linalg.norm(T)
    t0 = time.perf_counter()
    G = hotrg.gram(T)
    lam, U = hotrg.eigh_desc(G)
    w = U[:, :D].reshape(D, D, D)
    Tn = hotrg.hotrg_step(T, w)
    np.linalg.norm(Tn)
    dt = time.perf_counter() - t0
    return dt, step_flops(D, D, D)["total"]


def torch_fp64_step_seconds(D, dev, reps=1):
    """Comparator: one steady coarse-graining step (X = Y = X' = D) written in
    plain torch FP64 on the GPU -- einsum/tensordot contractions on cuBLAS
    DGEMM, torch.linalg.eigh (cuSOLVER) for the Gram matrix, Frobenius norm --
    timed with CUDA events after one warm-up.  Returns seconds per step."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    T = torch.randn((D, D, D, D), dtype=torch.float64, device=dev, generator=g)
    T /= torch.linalg.norm(T)
    yc = max(1, min(D, (1 << 27) // D ** 4))

    def step(T):
        A = torch.einsum("aiyj,ciyk->ajck", T, T)
        B = torch.einsum("bkjz,dkmz->bjdm", T, T)
        G = torch.einsum("ajck,bjdk->abcd", A, B).reshape(D * D, D * D)
        lam, U = torch.linalg.eigh(G)
        w = U[:, -D:].flip(-1).reshape(D, D, D)
        out = torch.empty((D, D, D, D), dtype=torch.float64, device=dev)
        for y0 in range(0, D, yc):
            Ty = T[:, :, y0:y0 + yc, :]                                   # [a, i, y, j]
            U1 = torch.tensordot(Ty, w, dims=([0], [0]))                  # [i, y, j, b, A]
            V = torch.tensordot(U1, T, dims=([3, 2], [0, 2]))             # [i, y, A, k, z]
            out[:, :, y0:y0 + yc, :] = torch.tensordot(V, w, dims=([0, 3], [0, 1])).permute(
                1, 3, 0, 2)                                               # [A, B, y, z]
        return out / torch.linalg.norm(out)

    step(T)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        step(T)
    b.record()
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / 1e3 / reps


def c1_latency(hot, reps=30):
    """C1: Ising beta = 0.44, D_cut = 8, 20 steps, FP64, forward + backward
    (ln Z/N and d(ln Z/N)/d beta) through the host-buffer C ABI; per-solve
    wall latency after warm-up."""
    lat = []
    with hot.Plan(2, 8, 20, "fp64") as p:
        for i in range(reps + 3):
            t0 = time.perf_counter()
            lnz, _, _ = p.forward_ising(0.44, 1.0, 0.0)
            _, db = p.backward(want_dbeta=True)
            if i >= 3:
                lat.append(time.perf_counter() - t0)
    lat = np.array(lat) * 1e3
    out = {"workload": "ising beta=0.44 d0=2 D_cut=8 20 steps, fp64, forward + backward",
           "solves": reps, "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "lnz_per_site": lnz, "dlnz_dbeta": db}
    g = golden("c1_ising")
    if g:
        out["abs_err_lnz_vs_oracle"] = abs(lnz - g["lnz"])
        out["rel_err_dbeta_vs_oracle"] = abs(db - g["dlnz_dbeta"]) / abs(g["dlnz_dbeta"])
    return out


def run_gemm_case(args):
    """One split-BF16 GEMM C = A B^T (three planes, accumulation chunks of
    128, the stage-2 kernel of the HOTRG step) of the given M, N, K on seeded
    N(0, 1) operands, through hotrg_gemm_split_check; checks a sample of C
    against FP64 and prints the kernel configuration.  Used as the small case
    of ncu captures of the stage-2 kernel."""
    import paper_1912_02780_gb300 as hot
    M, N, K = (int(x) for x in args.gemm_case.split(","))
    rng = np.random.default_rng(0)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = hot.gemm_split_check(A, B, planes=3, kchunk=2, cta_pair=args.stage2_pair > 0)
    rows = rng.integers(0, M, size=64)
    ref = A[rows] @ B.T
    err = float(np.max(np.abs(C[rows] - ref) / (np.abs(A[rows]) @ np.abs(B).T)))
    print(json.dumps({"gemm_case": [M, N, K], "planes": 3, "cta_pair": args.stage2_pair > 0,
                      "sampled_rel_err": err}), flush=True)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d0, d_cut, n, desc = WORKLOADS[args.workload]
    sched = schedule(d0, d_cut, n)
    total = sum(step_flops(*s)["total"] for s in sched)
    for _ in range(args.warmup):
        oracle_sample(d_cut)
    ts = []
    for _ in range(args.steps):
        dt, fl = oracle_sample(d_cut)
        ts.append(dt)
    t_step = float(np.mean(ts))
    solve_s = t_step * total / step_flops(d_cut, d_cut, d_cut)["total"]
    value = 1.0 / solve_s
    cores = os.cpu_count()
    sample = (f"one steady D={d_cut} coarse-graining step (Gram + FP64 eigh + contraction + norm) "
              f"per benchmark step, scaled to a {n}-step solve by useful flops")
    line = {"impl": "reference", "metric": "solves/s", "value": value, "unit": "solves/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_replay(hot, reqs, rate, slots, budget_gb, precision, split_from, srv=None):
    """Replay requests into the solve server in real time: request i arrives at
    its seeded Poisson time (synth.serving_stream, mean gap 1 / rate; rate =
    inf submits them all at once).  Latency = finish - submit on the server's
    clock.  Returns a dict of throughput and latency statistics."""
    own = srv is None
    if own:
        srv = hot.Server(int(budget_gb * 2 ** 30), slots)
    st0 = srv.stats()
    t0 = time.perf_counter()
    tickets = []
    base = reqs[0]["t_arrival"]
    for r in reqs:
        if np.isfinite(rate):
            # the stream's arrival times were drawn at rate 1: rescale
            dt = (r["t_arrival"] - base) / rate - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        tickets.append(srv.submit(r["beta"], r["J"], r["h"], r["d_cut"], r["n_steps"],
                                  r["want_grad"], precision, split_from))
    res = [srv.wait(t) for t in tickets]
    st = srv.stats()
    if own:
        srv.close()
    lat = np.array([x.t_finish - x.t_submit for x in res])
    svc = np.array([x.t_finish - x.t_start for x in res])
    span = max(x.t_finish for x in res) - min(x.t_submit for x in res)
    ok = sum(1 for x in res if x.status == 0)
    return {"requests": len(res), "ok": ok, "offered_rate": float(rate),
            "achieved_rate": ok / span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()),
            "service_time_mean_s": float(svc.mean()),
            "plans_created": st["plans_created"] - st0["plans_created"],
            "plans_evicted": st["plans_evicted"] - st0["plans_evicted"],
            "admission_waits": st["admission_waits"] - st0["admission_waits"],
            "peak_gb": st["peak_bytes"] / 2 ** 30}


def serving_stream_c5(n):
    """The C5 request mix at unit rate (beta ~ U[0.30, 0.60], h ~ U[0, 0.05],
    D_cut in {16, 24, 32, 48, 64}, n_steps in [20, 40], half with gradients)."""
    return synth.serving_stream(seed=2024, n=n, rate=1.0)


def serving_sample(hot, args, n_burst=16, n_rate=32, frac=0.25):
    """Short serving measurement for the default benchmark line: the first
    n_burst requests of the C5 stream submitted at once give a capacity
    (completed requests / makespan; this also builds the plans), then the next
    n_rate arrive as a Poisson stream at frac x that capacity.  A burst of a
    few requests overstates the sustained capacity (the stream's heavy
    requests -- D_cut = 64 with gradients -- are rare in it): the sustained
    rate under overload measured by --serve is about 0.3 of it."""
    stream = serving_stream_c5(n_burst + n_rate)
    srv = hot.Server(int(args.budget_gb * 2 ** 30), args.slots)
    burst = serve_replay(hot, stream[:n_burst], float("inf"), args.slots, args.budget_gb,
                         args.precision, args.split_from, srv)
    cap = burst["achieved_rate"]
    point = serve_replay(hot, stream[n_burst:], frac * cap, args.slots, args.budget_gb,
                         args.precision, args.split_from, srv)
    srv.close()
    return {"mix": "C5 (seed 2024): beta U[0.30,0.60], h U[0,0.05], D_cut {16,24,32,48,64}, "
                   "n_steps [20,40], half with gradients",
            "slots": args.slots, "budget_gb": args.budget_gb,
            "capacity_req_per_s": cap, "capacity_from": f"{n_burst} requests submitted at once",
            "rate_point": point,
            "note": f"p99 of {n_rate} requests (about their maximum); bench.py --serve runs "
                    f"longer rate sweeps"}


def run_serve(args):
    """Continuous-batching serving run on the C5 mix: the capacity from a burst
    of requests submitted at once, then Poisson streams at the given fractions
    of that capacity (--rates), --requests each, replayed in real time into
    the solve server; latency = finish - submit on the server's clock."""
    import paper_1912_02780_gb300 as hot
    fracs = [float(x) for x in args.rates.split(",")]
    n_burst = 16
    stream = serving_stream_c5(n_burst + args.requests * len(fracs))
    srv = hot.Server(int(args.budget_gb * 2 ** 30), args.slots)
    burst = serve_replay(hot, stream[:n_burst], float("inf"), args.slots, args.budget_gb,
                         args.precision, args.split_from, srv)
    cap = burst["achieved_rate"]
    points = []
    for i, fr in enumerate(fracs):
        reqs = stream[n_burst + i * args.requests:n_burst + (i + 1) * args.requests]
        pt = serve_replay(hot, reqs, fr * cap, args.slots, args.budget_gb, args.precision,
                          args.split_from, srv)
        pt["fraction_of_capacity"] = fr
        points.append(pt)
        print(json.dumps(pt), flush=True)
    srv.close()
    line = {"metric": "serving latency p50/p99 (s)", "unit": "s", "higher_is_better": False,
            "capacity_req_per_s": cap, "burst": burst, "points": points, "slots": args.slots,
            "budget_gb": args.budget_gb, "precision": args.precision,
            "split_from_step": args.split_from, "data": "synthetic",
            "config": {"workload": "ising serving stream (C5 mix)", "seed": 2024}}
    print(json.dumps(line), flush=True)


def run_grid(args):
    """The Ising beta grid (64 betas on [0.30, 0.60], D_cut = 32, 30 steps,
    forward + hand-written adjoint on one reused plan): ln Z/N, f, u and c
    (second-order finite differences of the adjoint's u), solves/s over the
    grid, and the largest errors against the oracle's stored grid."""
    import torch
    import paper_1912_02780_gb300 as hot  # noqa: F401  (loads the library)
    from paper_1912_02780_gb300.observables import ising_thermodynamics
    betas = synth.beta_grid()
    split = args.precision != "fp64"
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ising_thermodynamics(betas, 32, 30, args.precision,
                               split_from_step=args.split_from if split else 1,
                               hi_precision_steps=args.hi_steps, concurrent=args.concurrent,
                               sm_reserve=args.sm_reserve, grouped=args.grid_group)
    dt = time.perf_counter() - t0
    line = {"metric": "beta-grid solves/s (forward + backward)", "value": len(betas) / dt,
            "unit": "solves/s", "higher_is_better": True, "seconds": dt,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "c2_grid", "betas": len(betas), "d_cut": 32, "n_steps": 30,
                       "split_from_step": args.split_from if split else None,
                       "hi_precision_steps": args.hi_steps if split else None,
                       "concurrent_plans": args.concurrent, "sm_reserve": args.sm_reserve,
                       "grouped_forward": args.grid_group}}
    g = golden("c2_grid")
    if g:
        lnz_ref = np.array([q["lnz"] for q in g["points"]])
        u_ref = -np.array([q["dlnz_dbeta"] for q in g["points"]])
        line["max_abs_df_vs_oracle"] = float(np.max(np.abs(res["lnz"] - lnz_ref) / betas))
        line["max_rel_du_vs_oracle"] = float(np.max(np.abs(res["u"] - u_ref) / np.abs(u_ref)))
        # the oracle's specific heat by the same finite-difference rule
        from paper_1912_02780_gb300.observables import grid_derivative
        c_ref = -betas ** 2 * grid_derivative(betas, u_ref)
        line["max_rel_dc_vs_oracle"] = float(np.max(np.abs(res["c"] - c_ref) / np.abs(c_ref)))
    line["c_peak_beta"] = float(betas[int(np.argmax(res["c"]))])
    print(json.dumps(line), flush=True)


def run_dtrg_study(args):
    """Accuracy study of differentiable TRG near T_c (the shape of main text
    Fig. 2): Ising, D_cut = 24, 30 steps, split precision; HOTRG and dTRG
    (MERA updates with n_inner = 5 per layer, sweeps over the layers until a
    sweep changes ln Z/N by at most 1e-4 of the total improvement, at most
    --study-sweeps) free energies against Onsager on a beta scan across T_c."""
    from oracle import exact
    from paper_1912_02780_gb300.dtrg import dtrg_sweeps
    betas = [float(b) for b in args.study_betas.split(",")]
    rows = []
    for b in betas:
        t0 = time.perf_counter()
        r = dtrg_sweeps(2, 24, 30, n_sweeps=args.study_sweeps, n_inner=5, beta=b,
                        precision="bf16x6", split_from_step=5, tol=1e-4)
        ons = exact.onsager_lnz(b)
        row = {"beta": b, "rel_err_f_hotrg": abs(r["lnz_hotrg"] - ons) / abs(ons),
               "rel_err_f_dtrg": abs(r["lnz_final"] - ons) / abs(ons), "sweeps": r["sweeps"],
               "lnz_per_sweep": r["lnz"], "seconds": time.perf_counter() - t0}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"metric": "dTRG vs HOTRG free-energy error near T_c",
                      "config": {"model": "ising", "d_cut": 24, "n_steps": 30, "n_inner": 5,
                                 "tol": 1e-4, "precision": "bf16x6", "split_from_step": 5},
                      "rows": rows}), flush=True)


def run_dtrg(args):
    """Differentiable-TRG MERA updates at the workload's size: start from the
    HOTRG isometries, then time --steps updates (each a forward with the
    isometries as parameters, a backward with them fixed, and the SVD update of
    one steady-state layer) after --warmup untimed ones."""
    import torch
    import paper_1912_02780_gb300 as hot
    d0, d_cut, n, desc = WORKLOADS[args.workload]
    T0 = synth.random_symmetric_T0(0, d0)
    kw = dict(split_from_step=args.split_from, hi_precision_steps=args.hi_steps)
    with hot.Plan(d0, d_cut, n, args.precision, want_grad=True, **kw) as p0:
        lnz0, _, _ = p0.forward_tensor(T0)
        ws = p0.isometries()
    with hot.Plan(d0, d_cut, n, args.precision, want_grad=True, fixed_w_grad=True, w_given=True,
                  **kw) as p:
        p.set_isometries(ws)
        k0 = max(args.split_from + args.hi_steps, 2)    # steady-state layers
        layers = [k0 + i % (n - k0 + 1) for i in range(args.warmup + args.steps)]

        def update(k):
            p.forward_tensor(T0)
            p.backward()
            p.mera_update(k)

        for k in layers[:args.warmup]:
            update(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in layers[args.warmup:]:
            update(k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lnz1, _, _ = p.forward_tensor(T0)
    line = {"metric": "dTRG MERA updates/s", "value": args.steps / dt, "unit": "updates/s",
            "higher_is_better": True, "ms_per_update": 1e3 * dt / args.steps,
            "steps": args.steps, "warmup": args.warmup, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "layers": layers,
                       "split_from_step": args.split_from, "hi_precision_steps": args.hi_steps,
                       "update": "forward (isometries given) + backward (w fixed) + SVD of one layer"},
            "lnz_hotrg": lnz0, "lnz_after_updates": lnz1}
    print(json.dumps(line), flush=True)


def run_xy(args):
    """Scheme (b) on the infinite quantum XY chain, the workload of main text
    Fig. 3b: cool rho(tau), tau = 12.8 / 2^18 (second-order Trotter MPO), by
    17 doublings to beta = 12.8 (the exact final product doubles once more),
    per D_cut: plain scheme (b) and differentiable TRG with depth n_d (MERA
    updates of the newest layers against the free energy at the current
    temperature), wall time of the whole cooling and the free-energy error
    against the exact Jordan-Wigner solution."""
    import torch
    from oracle import xtrg as oxtrg
    from oracle import xy as oxy
    from paper_1912_02780_gb300 import xtrg as gx
    tau, n = 12.8 / 2 ** 18, 17
    beta_end = tau * 2 ** (n + 1)
    f_ex = -oxy.lnz_exact_infinite(beta_end) / beta_end
    ds = [int(x) for x in args.xy_d.split(",")]
    kw = dict(eigh_mode=1, eigh_power_iters=2)
    gx.cooling(tau, ds[0], 4, **kw)                      # warm-up (library load, first plans)
    rows = []
    for D in ds:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = gx.cooling(tau, D, n, **kw)
        t_plain = time.perf_counter() - t0
        row = {"d_cut": D, "seconds_plain": t_plain,
               "rel_err_f_plain": abs(plain["f"][-1] - f_ex) / abs(f_ex)}
        if args.xy_nd > 0:
            t0 = time.perf_counter()
            opt = gx.cooling(tau, D, n, n_d=args.xy_nd, n_sweeps=args.xy_sweeps,
                             n_inner=args.xy_inner, **kw)
            row["seconds_dtrg"] = time.perf_counter() - t0
            row["rel_err_f_dtrg"] = abs(opt["f"][-1] - f_ex) / abs(f_ex)
        rows.append(row)
        print(json.dumps(row), flush=True)
    cpu = None
    if not args.no_cpu_baseline:
        Dc = ds[0]
        t0 = time.perf_counter()
        oxtrg.xtrg_forward(oxy.mpo_cell(tau), Dc, n)
        cpu = {"d_cut": Dc, "seconds_plain": time.perf_counter() - t0, "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"plain scheme (b) cooling at D_cut = {Dc}"}
    fit = None
    big = [r for r in rows if r["d_cut"] >= 32]
    if len(big) >= 2:
        x = np.log([r["d_cut"] for r in big])
        y = np.log([r["seconds_plain"] for r in big])
        fit = float(np.polyfit(x, y, 1)[0])
    print(json.dumps({"metric": "XY-chain cooling to beta = 12.8, seconds per run",
                      "config": {"workload": "infinite XY chain, second-order Trotter MPO",
                                 "tau": tau, "doublings": n, "beta": beta_end,
                                 "dtrg": {"n_d": args.xy_nd, "n_sweeps": args.xy_sweeps,
                                          "n_inner": args.xy_inner},
                                 "eigensolver": "randomized subspace (2 power iterations, guard)",
                                 "precision": "fp64"},
                      "f_exact": f_ex, "rows": rows, "gamma_plain_fit_D>=32": fit,
                      "cpu_baseline": cpu}), flush=True)


def run_lbfgs(args):
    """L-BFGS optimisation of the isometries (SM Sec. D) against the MERA
    update: one sweep over the layers of the Ising network at beta = 0.40,
    D_cut = --lbfgs-d, 20 steps, FP64; wall time and the gain in ln Z/N
    against Onsager for each."""
    import torch
    from oracle import exact
    from paper_1912_02780_gb300 import dtrg as gd
    beta, D, n = 0.40, args.lbfgs_d, 20
    ons = exact.onsager_lnz(beta)
    gd.lbfgs_sweeps(2, D, 6, n_sweeps=1, n_iter=2, beta=beta)          # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lb = gd.lbfgs_sweeps(2, D, n, n_sweeps=1, n_iter=args.lbfgs_iters, beta=beta)
    t_lb = time.perf_counter() - t0
    t0 = time.perf_counter()
    me = gd.dtrg_sweeps(2, D, n, n_sweeps=1, n_inner=args.lbfgs_iters, beta=beta)
    t_me = time.perf_counter() - t0
    print(json.dumps({"metric": "isometry optimisation, one sweep",
                      "config": {"model": "ising", "beta": beta, "d_cut": D, "n_steps": n,
                                 "iterations_per_layer": args.lbfgs_iters, "precision": "fp64"},
                      "lbfgs": {"seconds": t_lb, "evaluations": lb["evals"],
                                "abs_err_lnz": abs(lb["lnz"][-1] - ons)},
                      "mera": {"seconds": t_me, "abs_err_lnz": abs(me["lnz_final"] - ons)},
                      "hotrg_abs_err_lnz": abs(lb["lnz_hotrg"] - ons)}), flush=True)


def run_group(args):
    """Grouped forward against the same solves one after another and on
    concurrent streams: G Ising solves (beta spread over [0.30, 0.60], h = 0)
    of one shape per D_cut, BF16X6 split from step 5, forward only, subspace
    eigensolver; the grouped forward with all plans on one stream and with
    each plan on its own stream (overlapping eigensolves); solves/s of each
    form and the launch counts; every result compared with the solo one (bit
    for bit)."""
    import torch
    import paper_1912_02780_gb300 as hot
    G, n = args.group_size, 30
    dev = torch.device("cuda", 0)
    betas = list(np.linspace(0.30, 0.60, G))
    rows = []
    for D in [int(x) for x in args.group_d.split(",")]:
        kw = dict(split_from_step=5, want_grad=False, hi_precision_steps=2, eigh_mode=1,
                  eigh_power_iters=2, eigh_warm_start=1)
        st = torch.cuda.Stream(dev)
        plans = [hot.Plan(2, D, n, "bf16x6", stream=st.cuda_stream, **kw) for _ in range(G)]
        grp = hot.Group(2, D, n, "bf16x6", max_count=G, stream=st.cuda_stream, **kw)
        streams = [torch.cuda.Stream(dev) for _ in range(G)]
        cplans = [hot.Plan(2, D, n, "bf16x6", stream=s2.cuda_stream, **kw) for s2 in streams]
        pool = ThreadPoolExecutor(max_workers=G)

        def solo():
            return [p.forward_ising(b)[0] for p, b in zip(plans, betas)]

        def grouped():
            return list(grp.forward_ising(plans, betas))

        def grouped_streams():
            return list(grp.forward_ising(cplans, betas))

        def concurrent():
            return list(pool.map(lambda i: cplans[i].forward_ising(betas[i])[0], range(G)))

        out = {"d_cut": D, "solves": G}
        ref = None
        for name, fn in (("solo", solo), ("grouped", grouped), ("concurrent", concurrent),
                         ("grouped_streams", grouped_streams)):
            for _ in range(args.warmup):
                r = fn()
            torch.cuda.synchronize()
            l0 = hot.kernel_launches()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                r = fn()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / args.steps
            out[name] = {"solves_per_s": G / dt, "ms": 1e3 * dt,
                         "launches_per_iteration": (hot.kernel_launches() - l0) // args.steps}
            if ref is None:
                ref = r
            else:
                out[name]["bit_identical_to_solo"] = bool(list(r) == list(ref))
        out["grouped_launches_total"] = grp.launches()
        rows.append(out)
        print(json.dumps(out), flush=True)
        pool.shutdown()
        grp.close()
        for p in plans + cplans:
            p.close()
    print(json.dumps({"metric": "grouped forward vs solo and concurrent solves",
                      "config": {"model": "ising", "n_steps": n, "solves": G,
                                 "precision": "bf16x6", "split_from_step": 5,
                                 "eigensolver": "subspace, warm start"},
                      "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4_d64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16x6", choices=["fp64", "bf16x3", "bf16x6"])
    ap.add_argument("--split-from", type=int, default=4)
    ap.add_argument("--hi-steps", type=int, default=3,
                    help="split steps (from --split-from) with four bf16 planes")
    ap.add_argument("--no-fp64-ref", action="store_true")
    ap.add_argument("--eigh-mode", type=int, default=1,
                    help="0: cuSOLVER partial eigensolve; 1: randomized subspace eigensolver")
    ap.add_argument("--power-iters", type=int, default=2)
    ap.add_argument("--eigh-block", type=int, default=0,
                    help="vectors in the subspace eigensolver's block (0: 4 D_cut)")
    ap.add_argument("--concurrent", type=int, default=3,
                    help="independent solves (seeds) per GPU per step, each on its own "
                         "stream, so that one solve's latency-bound FP64 eigensolve overlaps "
                         "the other's tensor-core stages (D_cut = 64, warm start, 16 SMs "
                         "reserved: 2 / 3 / 4 gave 0.619 / 0.629 / 0.603 solves/s)")
    ap.add_argument("--grad", type=int, default=0, help="1: each step is forward + backward")
    ap.add_argument("--n-steps", type=int, default=0,
                    help="override the workload's coarse-graining steps (profiling runs)")
    ap.add_argument("--split-chunk", type=int, default=0,
                    help="elements per plane of the split stage buffers (0: the library's "
                         "default; smaller = smaller plans and stage GEMMs, same results)")
    ap.add_argument("--stage2-group", type=int, default=0,
                    help="N-tiles per L2 raster group of the stage-2 GEMM (0: library default)")
    ap.add_argument("--stage2-pair", type=int, default=0,
                    help="stage-2 GEMM on CTA pairs (0: library default, 1: on, -1: off)")
    ap.add_argument("--sm-reserve", type=int, default=16,
                    help="SMs the contraction GEMMs of each plan leave to the other "
                         "concurrent solves' eigensolver kernels")
    ap.add_argument("--warm-start", type=int, default=1,
                    help="> 0: subspace eigensolver warm-started from step k-2 with this many "
                         "power iterations")
    ap.add_argument("--no-c1", action="store_true", help="skip the C1 latency measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: Poisson stream of Ising solves through the server")
    ap.add_argument("--grid", action="store_true",
                    help="the Ising beta grid (64 betas, D_cut = 32): f, u, c and solves/s")
    ap.add_argument("--dtrg", action="store_true",
                    help="time differentiable-TRG MERA updates at the workload's size")
    ap.add_argument("--dtrg-study", action="store_true",
                    help="dTRG vs HOTRG free-energy errors against Onsager near T_c (D_cut = 24)")
    ap.add_argument("--study-betas", default="0.40,0.42,0.43,0.4406867935097715,0.45,0.46,0.48")
    ap.add_argument("--study-sweeps", type=int, default=8)
    ap.add_argument("--xy", action="store_true",
                    help="scheme (b): XY-chain cooling to beta = 12.8, seconds per D_cut")
    ap.add_argument("--xy-d", default="16,32,64,96,128")
    ap.add_argument("--xy-nd", type=int, default=1, help="dTRG depth (0: plain only)")
    ap.add_argument("--xy-sweeps", type=int, default=1)
    ap.add_argument("--xy-inner", type=int, default=5)
    ap.add_argument("--lbfgs", action="store_true",
                    help="L-BFGS (exponential parametrisation) vs MERA update, one sweep")
    ap.add_argument("--lbfgs-d", type=int, default=16)
    ap.add_argument("--lbfgs-iters", type=int, default=5)
    ap.add_argument("--group", action="store_true",
                    help="grouped forward vs solo and concurrent solves at small D_cut")
    ap.add_argument("--group-d", default="16,24,32")
    ap.add_argument("--group-size", type=int, default=4)
    ap.add_argument("--grid-group", type=int, default=0,
                    help="--grid: betas per grouped forward (0: none)")
    ap.add_argument("--gemm-case", default="",
                    help="M,N,K: one three-plane split GEMM of the stage-2 kind through the "
                         "kernel-check entry point (a small case for ncu captures)")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0, help="offered requests per second")
    ap.add_argument("--rates", default="0.25,0.5,0.9",
                    help="--serve: offered load as fractions of the measured capacity")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the short serving measurement of the default run")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=240.0)
    args = ap.parse_args()
    if args.gemm_case:
        return run_gemm_case(args)
    if args.serve:
        return run_serve(args)
    if args.grid:
        return run_grid(args)
    if args.dtrg:
        return run_dtrg(args)
    if args.dtrg_study:
        return run_dtrg_study(args)
    if args.xy:
        return run_xy(args)
    if args.lbfgs:
        return run_lbfgs(args)
    if args.group:
        return run_group(args)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1912_02780_gb300 as hot

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    d0, d_cut, n, desc = WORKLOADS[args.workload]
    full_workload = True
    if args.n_steps and args.n_steps != n:
        # a shortened solve (profiling captures): no stored oracle value applies
        n, full_workload = args.n_steps, False
        desc += f" (shortened to {n} steps)"
    C = max(1, args.concurrent)
    # this rank's seeds (replicas on N GPUs take disjoint seed blocks)
    seeds = [rank * C + i for i in range(C)]
    T0s = [synth.random_symmetric_T0(sd, d0) for sd in seeds]
    streams = [torch.cuda.Stream(dev) for _ in range(C)]
    plans = [hot.Plan(d0, d_cut, n, args.precision, split_from_step=args.split_from,
                      want_grad=bool(args.grad), stream=st.cuda_stream,
                      hi_precision_steps=args.hi_steps, eigh_mode=args.eigh_mode,
                      eigh_power_iters=args.power_iters, eigh_block=args.eigh_block,
                      split_chunk_elems=args.split_chunk, stage2_n_group=args.stage2_group,
                      stage2_pair=args.stage2_pair, gemm_sm_reserve=args.sm_reserve,
                      eigh_warm_start=args.warm_start)
             for st in streams]
    T0_devs = [torch.tensor(t, dtype=torch.float64, device=dev) for t in T0s]
    out_devs = [torch.zeros(n + 2, dtype=torch.float64, device=dev) for _ in range(C)]
    grad_devs = [torch.zeros(d0 ** 4, dtype=torch.float64, device=dev) for _ in range(C)]
    pool = ThreadPoolExecutor(max_workers=C)

    def solve_dev(i):
        plans[i].forward_device(T0_devs[i].data_ptr(), out_devs[i].data_ptr())
        if args.grad:
            plans[i].backward_device(grad_devs[i].data_ptr())
        plans[i].sync()

    def batch(fn):
        # one benchmark step: the C solves of this rank, each driven by its own
        # host thread on its own stream, so that they overlap on the device
        list(pool.map(fn, range(C)))

    for _ in range(args.warmup):
        batch(solve_dev)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()

    sampler = ClockSampler(local if world > 1 else 0)
    sampler.start()
    launches0 = hot.kernel_launches()
    main_stream = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(main_stream)
    for st in streams:
        st.wait_event(ev0)
    for _ in range(args.steps):
        batch(solve_dev)
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        main_stream.wait_event(e)
    ev1.record(main_stream)
    torch.cuda.synchronize(dev)
    launches = hot.kernel_launches() - launches0
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total, solves = aggregate_over_ranks(ms_total, args.steps * C, dist, dev)
    if dist:
        dist.barrier()
    ms_per_step = ms_total / args.steps
    value = solves / (ms_total / 1e3)
    lnzs = [float(o[0].item()) for o in out_devs]

    guard = [pl.eigh_diagnostics() for pl in plans]

    # one solve alone with per-stage CUDA events on its stream: stage breakdown
    # and the roofline of the stage-2 kernel (not overlapped with other solves).
    # Timed twice: with the timed region's plan (its contraction GEMMs leave
    # --sm-reserve SMs to the other solves) and with a plan whose GEMMs use
    # every SM, which is the kernel's own roofline.
    def profiled_solve(plan, i):
        plan.profile(True)
        t_a = torch.cuda.Event(enable_timing=True)
        t_b = torch.cuda.Event(enable_timing=True)
        t_a.record(streams[i])
        plan.forward_device(T0_devs[i].data_ptr(), out_devs[i].data_ptr())
        if args.grad:
            plan.backward_device(grad_devs[i].data_ptr())
        plan.sync()
        t_b.record(streams[i])
        torch.cuda.synchronize(dev)
        pr = plan.profile_read()
        plan.profile(False)
        return pr, t_a.elapsed_time(t_b)

    prof_bench, single_ms_bench = profiled_solve(plans[0], 0)
    prof, single_ms = prof_bench, single_ms_bench
    if args.sm_reserve > 0:
        with hot.Plan(d0, d_cut, n, args.precision, split_from_step=args.split_from,
                      want_grad=bool(args.grad), stream=streams[0].cuda_stream,
                      hi_precision_steps=args.hi_steps, eigh_mode=args.eigh_mode,
                      eigh_power_iters=args.power_iters, eigh_block=args.eigh_block,
                      split_chunk_elems=args.split_chunk, stage2_n_group=args.stage2_group,
                      stage2_pair=args.stage2_pair, gemm_sm_reserve=0,
                      eigh_warm_start=args.warm_start) as pfull:
            pfull.forward_device(T0_devs[0].data_ptr(), out_devs[0].data_ptr())
            pfull.sync()
            prof, single_ms = profiled_solve(pfull, 0)

    # useful / executed flops of one solve and of the stage-2 launches
    sched = schedule(d0, d_cut, n)
    npairs = {"fp64": 1, "bf16x3": 3, "bf16x6": 6}[args.precision]
    useful = 0.0
    executed_tc = 0.0
    s2_tc_useful = 0.0      # stage-2 launches of the three-plane steps (profile slot "s2")
    for k, (X, Y, Xp) in enumerate(sched, start=1):
        f = step_flops(X, Y, Xp)
        useful += f["total"]
        if is_split_step(k, X, Y, Xp, args.split_from, args.precision):
            nprod = products_of_step(k, args.split_from, args.hi_steps, args.precision)
            executed_tc += f["total"] * nprod
            if nprod == npairs:
                s2_tc_useful += f["s2"]
    bwd_factor = 4.0 if args.grad else 1.0   # backward ~3x forward incl. recompute
    useful_tflops = useful * bwd_factor * solves / (ms_total / 1e3) / 1e12

    peaks = measured_peaks()
    roof = None
    if "s2" in prof and s2_tc_useful > 0:
        s2_ms, s2_launches = prof["s2"]
        s2_ms_per_launch = s2_ms / s2_launches
        exec_per_launch = s2_tc_useful * npairs / s2_launches
        achieved = exec_per_launch / (s2_ms_per_launch / 1e3) / 1e12
        if peaks:
            peak, src = peaks.get("bf16_tflops_sustained"), "measured (sustained)"
        else:
            peak, src = 1700.0, "fallback (sustained)"
        traffic = None
        if (STAGE2_TRAFFIC["gemm_tc_sha256"] == gemm_source_sha() and d_cut == 64
                and STAGE2_TRAFFIC["bytes_per_launch_d64"]):
            traffic = STAGE2_TRAFFIC["bytes_per_launch_d64"]
        in_bench = None
        if "s2" in prof_bench and args.sm_reserve > 0:
            b_ms = prof_bench["s2"][0] / prof_bench["s2"][1]
            b_ach = exec_per_launch / (b_ms / 1e3) / 1e12
            ctas = 152 - args.sm_reserve
            in_bench = {"ctas": ctas, "ms_per_launch": b_ms, "achieved": b_ach,
                        "frac_of_peak_scaled_to_ctas": b_ach / (peak * ctas / 152) if peak else None}
        roof = {"kernel": "tc_gemm_kernel<128,3> (stage 2, O(D^7), three-plane steps)",
                "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "peak_source": src,
                "traffic": traffic,
                "useful_per_launch_tflop": s2_tc_useful / s2_launches / 1e12,
                "executed_per_launch_tflop": exec_per_launch / 1e12,
                "ms_per_launch": s2_ms_per_launch,
                "timed": "CUDA events around every stage-2 launch of one solve run alone, "
                         "its GEMMs on every SM",
                "in_timed_region_config": in_bench}

    line = {"metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "d0": d0, "d_cut": d_cut,
                       "n_steps": n, "precision": args.precision,
                       "split_from_step": args.split_from, "hi_precision_steps": args.hi_steps,
                       "split_chunk_elems": args.split_chunk or "default (2^30)",
                       "eigh": ("randomized subspace, block %d, %d power iterations"
                                % (args.eigh_block or 4 * d_cut, args.power_iters)
                                if args.eigh_mode == 1 else "cuSOLVER syevdx (top D'+1)"),
                       "grad": bool(args.grad), "solves_per_step": C,
                       "seeds": seeds,
                       "l2": "working set > L2 (D^5 intermediates of several GB per step)",
                       "parallelism": f"replicas x{world}, {C} concurrent solves per GPU"},
            "useful_tflops": useful_tflops,
            "executed_tc_tflop_per_solve": executed_tc / 1e12,
            "single_solve_ms": single_ms,
            "single_solve_ms_timed_config": single_ms_bench,
            "lnz_per_site": lnzs,
            "stage_ms_per_solve": {k: v[0] for k, v in prof.items()},
            "gpu_launches": int(launches),
            "eigh_guard": {"bound": "2^-k r_k <= 1e-9 (r_k: relative residual of the kept "
                                    "Ritz pairs at step k), else up to four more power "
                                    "iterations, then the exact eigensolver",
                           "max_residual": [float(np.nanmax(g_[0])) if np.any(np.isfinite(g_[0]))
                                            else None for g_ in guard],
                           "extra_iters": [int(g_[1].sum()) for g_ in guard],
                           "exact_steps": [int(g_[2].sum()) for g_ in guard],
                           "guard_steps_total": [g_[3] for g_ in guard]},
            "clocks": clocks}
    if roof:
        line["roofline"] = roof
    if rank == 0 and not args.grad and full_workload:
        errs = {}
        for sd, lz in zip(seeds, lnzs):
            g = golden(f"{args.workload}_s{sd}")
            if g:
                errs[f"seed{sd}"] = abs(lz - g["lnz"])
        if errs:
            line["abs_err_lnz_vs_oracle"] = errs

    # end to end through the host-buffer C ABI (pinned host input, host results)
    if not args.no_e2e and rank == 0:
        T0_pins = [torch.tensor(t, dtype=torch.float64).pin_memory().numpy() for t in T0s]

        def solve_host(i):
            plans[i].forward_tensor(T0_pins[i])
            if args.grad:
                plans[i].backward()

        batch(solve_host)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main_stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            batch(solve_host)
        torch.cuda.synchronize(dev)
        e1.record(main_stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        e2e_ms = max(e0.elapsed_time(e1), wall * 1e3)
        line["e2e"] = {"value": args.steps * C / (e2e_ms / 1e3), "unit": "solves/s",
                       "h2d_bytes_per_step": C * T0s[0].nbytes,
                       "d2h_bytes_per_step": C * (8 * (n + 2) + (T0s[0].nbytes if args.grad else 0))}

    # the plain FP64-on-GPU form of the same solve: one steady step timed (an
    # FP64 plan of `first` steps minus one of first - 1 steps), scaled to the solve
    if rank == 0 and world == 1 and not args.no_fp64_ref and args.precision != "fp64":
        def fp64_time(nsteps):
            with hot.Plan(d0, d_cut, nsteps, "fp64", want_grad=False,
                          stream=streams[0].cuda_stream) as p64:
                p64.forward_device(T0_devs[0].data_ptr(), out_devs[0].data_ptr())
                p64.sync()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(streams[0])
                p64.forward_device(T0_devs[0].data_ptr(), out_devs[0].data_ptr())
                b.record(streams[0])
                p64.sync()
                return a.elapsed_time(b) / 1e3
        first = next(k for k, s_ in enumerate(sched, start=1) if s_ == (d_cut, d_cut, d_cut))
        t_lo, t_hi = fp64_time(first - 1), fp64_time(first)
        steady = t_hi - t_lo
        t_solve = t_lo + steady * (n - first + 1)
        # the same steady step as plain torch FP64 (cuBLAS DGEMM + cuSOLVER eigh)
        steady_torch = torch_fp64_step_seconds(d_cut, dev)
        t_solve_torch = t_lo + steady_torch * (n - first + 1)
        best = min(t_solve, t_solve_torch)
        line["fp64_gpu"] = {"solves_per_s": 1.0 / best,
                            "library_fp64_solves_per_s": 1.0 / t_solve,
                            "library_fp64_steady_step_s": steady,
                            "torch_fp64_solves_per_s": 1.0 / t_solve_torch,
                            "torch_fp64_steady_step_s": steady_torch,
                            "speedup_of_split": value * best,
                            "speedup_single_solve": (1e3 / single_ms) * best,
                            "how": f"the faster of two FP64-on-GPU forms: this library's FP64 "
                                   f"plans of {first - 1} and {first} steps timed with CUDA "
                                   f"events (steady step = the difference), and one steady "
                                   f"step in plain torch FP64 (einsum/tensordot on cuBLAS "
                                   f"DGEMM, torch.linalg.eigh); solve = the first "
                                   f"{first - 1} steps + {n - first + 1} steady steps"}

    if rank == 0 and not args.no_c1:
        line["c1_latency"] = c1_latency(hot)

    if rank == 0 and world == 1 and not args.no_serving:
        # the other solves' plans are released first: the server has the device
        pool.shutdown()
        for p_ in plans:
            p_.close()
        plans = []
        torch.cuda.synchronize(dev)
        line["serving"] = serving_sample(hot, args)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, fl = oracle_sample(d_cut)
        total = sum(step_flops(*s)["total"] for s in sched)
        cpu_solve_s = dt * total / fl
        line["cpu_baseline"] = {
            "value": 1.0 / cpu_solve_s, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"one steady D={d_cut} step of the FP64 NumPy/LAPACK oracle ({dt:.1f} s), "
                       f"scaled to the {n}-step solve by useful flops")}
    pool.shutdown()
    for p_ in plans:
        p_.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
