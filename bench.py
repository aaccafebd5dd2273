#!/usr/bin/env python
"""Throughput benchmark of the SGN constraint-solve hot path on GB300.

Workload (default): a batched ensemble of 256 independent 1d periodic SGN instances,
n = 2^k with k ~ U{9..13} (seed 2506 + rank), L = 200, g = 9.81, a solitary wave
(a ~ U[0.05, 0.4]) approaching a tanh shelf (start ~ U[0.3L, 0.7L], depth ratio
~ U[0.4, 0.8], ramps of width 5, length 0.4L), per-instance dt = 0.25 dx / sqrt(g(1+a)).
One bench step = one RK4 step of every instance (Eq:ERK: 4 right-hand sides, 4 PCG
constraint solves with the preconditioner A, coefficient reductions, stage sums), mixed
precision (float32 inner PCG inside float64 refinement), rtol 1e-10.

Metric: grid-point-steps/s = sum_i n_i * steps / seconds.  The line also reports the
batched float64 form, the plain float64 one-instance-per-launch form, the error against
float64, an end-to-end number through host buffers, the roofline of the dominant kernel
and the CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SGN grid-point-steps/s batched vs plain at ≤1e-6 rel err; p50/p99 solve ms"
UNIT = "grid-point-steps/s"
FP32_PEAK = 152 * 128 * 2 * 2.07e9          # FMA lanes x 2 flops x max SM clock
FP64_PEAK = 1.2e12                          # measured FMA throughput on this part
RTOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        pg = dist
    return world, rank, local, pg


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                       "-lms", "200", "-i", str(self.device)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------
# CPU oracle baseline (also the --impl reference arm)
# --------------------------------------------------------------------------------------

def oracle_sample(ens, seconds):
    """RK4 steps of the oracle over instances of the ensemble until `seconds` elapse."""
    from oracle import sgn_oracle as O
    done_pts, t_used, results = 0, 0.0, []
    order = sorted(range(len(ens)), key=lambda i: ens[i].n)
    pick = order[:: max(1, len(order) // 16)]
    for i in pick:
        c = ens[i]
        grid = O.make_grid(1, c.n, c.L, c.g)
        st = O.init_state(c.eta, c.u, c.h, grid)
        t0 = time.perf_counter()
        O.rk4_step(st, c.dt, RTOL)
        t_used += time.perf_counter() - t0
        done_pts += c.n
        results.append((i, st.eta.copy(), st.u.copy()))
        if t_used > seconds:
            break
    return done_pts, t_used, results


def reference_arm(args):
    from paper_2506_16045_gb300 import inputs as I
    ens = I.ensemble_1d(count=args.count, seed=2506)
    vals = []
    per_step = max(1.0, min(args.cpu_seconds, 20.0) / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(ens, 0.2)
    for _ in range(args.steps):
        pts, t, _ = oracle_sample(ens, per_step)
        vals.append((pts, t))
    pts = sum(p for p, _ in vals)
    tt = sum(t for _, t in vals)
    value = pts / tt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "ensemble256-1d-rk4", "instances": args.count,
                   "sample": "oracle RK4 steps on a size-stratified subset of the ensemble"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{pts} instance-points over {args.steps} bounded steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------

class Ensemble:
    def __init__(self, sgn, ctx, ens, torch):
        import numpy as np
        self.sgn, self.ctx, self.ens, self.torch = sgn, ctx, ens, torch
        self.lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in ens])
        cat = lambda k: np.concatenate([getattr(c, k) for c in ens])
        dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
        self.eta0, self.u0, self.h = dev(cat("eta")), dev(cat("u")), dev(cat("h"))
        self.eta = self.eta0.clone()
        self.u = self.u0.clone()
        self.U = torch.zeros_like(self.eta)
        self.gh = torch.zeros_like(self.eta)
        self.st = sgn.State(self.lay, self.eta, self.U, self.u, self.h, self.gh)
        self.dts = [c.dt for c in ens]
        self.points = int(sum(c.n for c in ens))
        self.classes = sorted({c.n for c in ens})

    def reset(self):
        self.eta.copy_(self.eta0)
        self.u.copy_(self.u0)
        self.st.init()

    def step(self, prec, n=1):
        self.st.rk4(self.dts, n, rtol=RTOL, maxit=4000, prec=prec)

    def launches_per_step(self):
        c = len(self.classes)
        return 4 * c + 4 * c + 8 + 4          # rhs, pcg per size class; stage sums; counters


def gpu_arm(args, world, rank, local, pg):
    import numpy as np
    import torch

    from paper_2506_16045_gb300 import inputs as I
    from paper_2506_16045_gb300 import sgn

    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    sgn.load()
    ctx = sgn.Context(dev_index)
    ens = I.ensemble_1d(count=args.count, seed=2506 + rank)
    E = Ensemble(sgn, ctx, ens, torch)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()

    # ---- mixed precision, batched (the headline)
    E.reset()
    for _ in range(args.warmup):
        E.step(sgn.PREC_MIXED)
    torch.cuda.synchronize()
    s0 = E.st.stats()
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    with Clocks(dev_index) as clk:
        for k in range(args.steps):
            flush.add_(1.0)
            ev[k][0].record(stream)
            E.step(sgn.PREC_MIXED)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    ctx.profile(False)
    prof = ctx.profile_read()
    s1 = E.st.stats()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = sum(step_ms)
    eta_mixed = E.eta.cpu().numpy().copy()
    u_mixed = E.u.cpu().numpy().copy()
    if pg is not None:
        import torch.distributed as dist
        tt = torch.tensor([t_ms], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt[0])
        pts = torch.tensor([float(E.points)], dtype=torch.float64)
        dist.all_reduce(pts, op=dist.ReduceOp.SUM)
        total_points = float(pts[0])
    else:
        total_points = float(E.points)
    value = total_points * args.steps / (t_ms * 1e-3)

    # ---- float64 batched from the same start: accuracy reference and the batched-fp64 rate
    E.reset()
    nref = args.warmup + args.steps
    E.step(sgn.PREC_FP64, max(0, nref - 2))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    flush.add_(1.0)
    e0.record(stream)
    E.step(sgn.PREC_FP64, min(2, nref))
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1) / min(2, nref)
    eta64 = E.eta.cpu().numpy()
    u64 = E.u.cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    err_eta, err_u = rel(eta_mixed, eta64), rel(u_mixed, u64)
    zeta64 = eta64 - E.h.cpu().numpy()
    err_zeta = rel(eta_mixed - E.h.cpu().numpy(), zeta64)

    # ---- plain float64, one instance per launch, on a size-stratified sample
    plain = None
    if not args.no_plain:
        order = sorted(range(len(ens)), key=lambda i: ens[i].n)
        pick = order[:: max(1, len(order) // 16)]
        pts, tms = 0, 0.0
        for i in pick:
            E1 = Ensemble(sgn, ctx, [ens[i]], torch)
            E1.reset()
            E1.step(sgn.PREC_FP64)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            E1.step(sgn.PREC_FP64)
            b.record(stream)
            torch.cuda.synchronize()
            tms += a.elapsed_time(b)
            pts += ens[i].n
            E1.st.close()
        plain = {"value": pts / (tms * 1e-3), "unit": UNIT,
                 "sample": f"{len(pick)} size-stratified instances, 1 RK4 step each, one "
                           "instance per launch"}

    # ---- end to end through host buffers: H2D of the state, one step, D2H of (eta, u)
    E.reset()
    torch.cuda.synchronize()
    P = E.points
    h_eta = torch.empty(P, dtype=torch.float64, pin_memory=True)
    h_U = torch.empty(P, dtype=torch.float64, pin_memory=True)
    h_u = torch.empty(P, dtype=torch.float64, pin_memory=True)
    h_eta.copy_(E.eta)
    h_U.copy_(E.U)
    h_u.copy_(E.u)
    ke = min(args.steps, 5)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(ke):
        E.eta.copy_(h_eta, non_blocking=True)
        E.U.copy_(h_U, non_blocking=True)
        E.u.copy_(h_u, non_blocking=True)
        E.step(sgn.PREC_MIXED)
        h_eta.copy_(E.eta, non_blocking=True)
        h_u.copy_(E.u, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / ke

    # ---- CPU oracle on a bounded sample (rank 0, N = 1) and its agreement after 1 step
    cpu = None
    oracle_err = None
    if rank == 0 and world == 1:
        pts, t_cpu, res = oracle_sample(ens, args.cpu_seconds)
        cpu = {"value": pts / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(res)} size-stratified instances x 1 RK4 step ({pts} points), "
                         f"numpy float64, {t_cpu:.1f} s"}
        E.reset()
        E.step(sgn.PREC_MIXED)
        eg, ug = E.eta.cpu().numpy(), E.u.cpu().numpy()
        offs = E.lay.offsets
        num = den = 0.0
        for i, oe, ou in res:
            num += np.sum((eg[offs[i]:offs[i + 1]] - oe) ** 2) + np.sum((ug[offs[i]:offs[i + 1]] - ou) ** 2)
            den += np.sum(oe ** 2) + np.sum(ou ** 2)
        oracle_err = math.sqrt(num / den)

    # ---- roofline of the dominant kernel (the PCG launch groups, timed in the region)
    f32 = s1["flops32"] - s0["flops32"]
    f64 = s1["flops64"] - s0["flops64"]
    pcg_s = prof["pcg_ms"] * 1e-3
    t_min = f32 / FP32_PEAK + f64 / FP64_PEAK
    achieved = (f32 + f64 * FP32_PEAK / FP64_PEAK) / pcg_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
            "frac": t_min / pcg_s, "traffic": None,
            "kernel": "k_pcg1d<float,...,mixed> (one launch per size class per solve)",
            "note": "fp32-equivalent: float64 flops weighted by the fp32/fp64 peak ratio",
            "pcg_share_of_step": prof["pcg_ms"] / t_ms, "rhs_share_of_step": prof["rhs_ms"] / t_ms}

    srt = sorted(step_ms)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble256-1d-rk4: 256 uneven 1d shelf instances, n in "
                               "{512..8192}, RK4 + mixed PCG, rtol 1e-10",
                   "instances": args.count, "points_per_gpu": E.points, "scheme": "RK4",
                   "precision": "mixed (f32 inner PCG, f64 refinement/dots/stage sums/RHS)",
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas"},
        "e2e": {"value": total_points / (e2e_ms * 1e-3) if world == 1 else None, "unit": UNIT,
                "h2d_bytes_per_step": 3 * 8 * P, "d2h_bytes_per_step": 2 * 8 * P},
        "gpu_launches": E.launches_per_step() * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "cpu_baseline": cpu,
        "accuracy": {"rel_l2_eta_vs_fp64": err_eta, "rel_l2_u_vs_fp64": err_u,
                     "rel_l2_zeta_vs_fp64": err_zeta, "steps_compared": nref,
                     "rel_l2_vs_oracle_sample_1step": oracle_err},
        "batched_fp64": {"value": total_points / (fp64_ms * 1e-3), "unit": UNIT},
        "plain_fp64": plain,
        "step_latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1,
                                                                     int(0.99 * len(srt)))]},
        "solver": {"solves": s1["solves"] - s0["solves"],
                   "iterations": s1["iterations"] - s0["iterations"],
                   "max_iters": s1["max_iters"], "status": s1["status"]},
    }
    if rank == 0:
        print(json.dumps(line))
    E.st.close()


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    gpu_arm(args, world, rank, local, pg)


if __name__ == "__main__":
    main()
