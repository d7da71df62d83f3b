"""Benchmark of the HOTRG hot path on GB300.

Workload (default): the split-precision configuration of the headline metric,
a seeded random reflection-symmetric rank-4 tensor T0 (bond dimension 4,
entries N(0,1), max|T| = 1), D_cut = 64, 30 coarse-graining steps, the O(D^7)
contractions and the Gram matrices on the tensor cores in three-plane split
BF16 (FP32 accumulation flushed every 64-wide K slab into compensated sums),
the eigensolve, norms and log-norm accumulation in FP64; steps before
--split-from run entirely in FP64.  One benchmark step = one complete solve
(forward; with --grad also the backward).

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


def run_serve(args):
    """Continuous-batching serving run: seeded Poisson arrivals of Ising solves
    (beta ~ U[0.30, 0.60], h ~ U[0, 0.05], D_cut in {16, 24, 32, 48, 64},
    n_steps in [20, 40], half of them with gradients), replayed in real time
    into the solve server; latency = finish - submit on the server's clock."""
    import paper_1912_02780_gb300 as hot
    stream = synth.serving_stream(seed=2024, n=args.requests, rate=args.rate)
    srv = hot.Server(int(args.budget_gb * 2 ** 30), args.slots)
    t0 = time.perf_counter()
    tickets = []
    for r in stream:
        dt = r["t_arrival"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(r["beta"], r["J"], r["h"], r["d_cut"], r["n_steps"],
                                  r["want_grad"], args.precision, args.split_from))
    res = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    lat = np.array([x.t_finish - x.t_submit for x in res])
    svc = np.array([x.t_finish - x.t_start for x in res])
    span = max(x.t_finish for x in res) - min(x.t_submit for x in res)
    ok = sum(1 for x in res if x.status == 0)
    line = {"metric": "serving latency p50/p99 (s)", "value": float(np.percentile(lat, 50)),
            "p99": float(np.percentile(lat, 99)), "unit": "s", "higher_is_better": False,
            "solves_per_s": ok / span, "offered_rate": args.rate,
            "achieved_rate": ok / span, "requests": len(res), "ok": ok,
            "service_time_mean_s": float(svc.mean()), "slots": args.slots,
            "budget_gb": args.budget_gb, "peak_gb": st["peak_bytes"] / 2 ** 30,
            "plans_created": st["plans_created"], "plans_evicted": st["plans_evicted"],
            "precision": args.precision, "split_from_step": args.split_from,
            "data": "synthetic", "config": {"workload": "ising serving stream", "seed": 2024}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4_d64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16x6", choices=["fp64", "bf16x3", "bf16x6"])
    ap.add_argument("--split-from", type=int, default=5)
    ap.add_argument("--grad", type=int, default=0, help="1: each step is forward + backward")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: Poisson stream of Ising solves through the server")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0, help="offered requests per second")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    args = ap.parse_args()
    if args.serve:
        return run_serve(args)
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
    T0 = synth.random_symmetric_T0(rank if world > 1 else 0, d0)
    stream = torch.cuda.current_stream(dev)
    plan = hot.Plan(d0, d_cut, n, args.precision, split_from_step=args.split_from,
                    want_grad=bool(args.grad), stream=stream.cuda_stream)
    T0_dev = torch.tensor(T0, dtype=torch.float64, device=dev)
    out_dev = torch.zeros(n + 2, dtype=torch.float64, device=dev)
    grad_dev = torch.zeros(d0 ** 4, dtype=torch.float64, device=dev)

    def one_solve():
        plan.forward_device(T0_dev.data_ptr(), out_dev.data_ptr())
        if args.grad:
            plan.backward_device(grad_dev.data_ptr())

    for _ in range(args.warmup):
        one_solve()
    plan.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local if world > 1 else 0)
    sampler.start()
    plan.profile(True)
    launches0 = hot.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        one_solve()
    ev1.record(stream)
    plan.sync()
    torch.cuda.synchronize(dev)
    launches = hot.kernel_launches() - launches0
    clocks = sampler.stop()
    prof = plan.profile_read()
    plan.profile(False)
    ms_total = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    ms_per_step = ms_total / args.steps
    solves = args.steps * world
    value = solves / (ms_total / 1e3)

    res = out_dev.cpu().numpy()
    lnz = float(res[0])

    # useful / executed flops of one solve and of the stage-2 launches
    sched = schedule(d0, d_cut, n)
    npairs = {"fp64": 1, "bf16x3": 3, "bf16x6": 6}[args.precision]
    useful = 0.0
    executed_tc = 0.0
    s2_tc_useful = 0.0
    for k, (X, Y, Xp) in enumerate(sched, start=1):
        f = step_flops(X, Y, Xp)
        useful += f["total"]
        if is_split_step(k, X, Y, Xp, args.split_from, args.precision):
            executed_tc += f["total"] * npairs
            s2_tc_useful += f["s2"]
    bwd_factor = 4.0 if args.grad else 1.0   # backward ~3x forward incl. recompute
    useful_tflops = useful * bwd_factor * args.steps / (ms_total / 1e3) / 1e12

    peaks = measured_peaks()
    roof = None
    if "s2" in prof and s2_tc_useful > 0:
        s2_ms, s2_launches = prof["s2"]
        s2_ms_per_launch = s2_ms / s2_launches
        exec_per_launch = s2_tc_useful * npairs * args.steps / s2_launches
        achieved = exec_per_launch / (s2_ms_per_launch / 1e3) / 1e12
        if peaks:
            peak, src = peaks.get("bf16_tflops_sustained"), "measured (sustained)"
        else:
            peak, src = 1700.0, "fallback (sustained)"
        roof = {"kernel": "tc_gemm_kernel (stage 2, O(D^7))", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "peak_source": src,
                "traffic": None,
                "useful_per_launch_tflop": s2_tc_useful * args.steps / s2_launches / 1e12,
                "executed_per_launch_tflop": exec_per_launch / 1e12,
                "ms_per_launch": s2_ms_per_launch}

    line = {"metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "d0": d0, "d_cut": d_cut,
                       "n_steps": n, "precision": args.precision,
                       "split_from_step": args.split_from, "grad": bool(args.grad),
                       "l2": "working set > L2 (D^5 intermediates of several GB per step)",
                       "parallelism": f"replicas x{world}"},
            "useful_tflops": useful_tflops,
            "executed_tc_tflop_per_solve": executed_tc / 1e12,
            "lnz_per_site": lnz,
            "stage_ms_per_solve": {k: v[0] / args.steps for k, v in prof.items()},
            "gpu_launches": int(launches),
            "clocks": clocks}
    if roof:
        line["roofline"] = roof
    g = golden(f"{args.workload}_s0") if rank == 0 else None
    if g and not args.grad and world == 1:
        line["abs_err_lnz_vs_oracle"] = abs(lnz - g["lnz"])

    # end to end through the host-buffer C ABI (pinned host input, host results)
    if not args.no_e2e and rank == 0:
        T0_pin = torch.tensor(T0, dtype=torch.float64).pin_memory()
        T0_np = T0_pin.numpy()
        for _ in range(1):
            plan.forward_tensor(T0_np)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.forward_tensor(T0_np)
            if args.grad:
                plan.backward()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        e2e_ms = max(e0.elapsed_time(e1), wall * 1e3)
        line["e2e"] = {"value": args.steps / (e2e_ms / 1e3), "unit": "solves/s",
                       "h2d_bytes_per_step": T0.nbytes,
                       "d2h_bytes_per_step": 8 * (n + 2) + (T0.nbytes if args.grad else 0)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, fl = oracle_sample(d_cut)
        total = sum(step_flops(*s)["total"] for s in sched)
        cpu_solve_s = dt * total / fl
        line["cpu_baseline"] = {
            "value": 1.0 / cpu_solve_s, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"one steady D={d_cut} step of the FP64 NumPy/LAPACK oracle ({dt:.1f} s), "
                       f"scaled to the {n}-step solve by useful flops")}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
