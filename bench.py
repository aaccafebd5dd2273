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
FULL_STEPS = 200            # the ensemble configuration's run length
FP32_PEAK = 152 * 128 * 2 * 2.07e9          # FMA lanes x 2 flops x max SM clock
# float32 FMA rate of a dependent-chain probe kernel measured on the GB300s (TFLOP/s)
FP32_PROBE_TFLOPS = 75.3
# DRAM bytes (read + write) per launch of the 2d persistent inner-solve kernel on the
# pcg2d_batch configuration (16 instances of 512^2), from an ncu capture of this kernel
# version, the staged form with split transform addresses (dram__bytes_read.sum +
# dram__bytes_write.sum, the mean of the first solve's two launches: 4.368e9 and 6.134e9
# bytes)
PCG2D_TRAFFIC_BYTES = 5.251e9


def hbm_peak():
    """The measured HBM copy bandwidth (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"
# float32 operations per double-float flop in a complex FFT butterfly: a double-float add is
# 11 float32 operations and a multiply 7, so a butterfly costs about 9.6 times its float32 form
DF_COST = 9.6
RTOL = 1e-10
# What the mixed path computes in which arithmetic (the line's accuracy block gives the
# measured effect against the float64 path and the oracle)
PRECISION_MIXED = ("mixed: float32 inner PCG (FFTs, matvecs, Krylov vectors; float32 "
                   "per-thread dot partials reduced across the CTA in double-float); refinement "
                   "residual b - G x and its dot r.A^-1 r in double-float (pairs of float32, "
                   "~48-bit significand); right-hand side in double-float (2d: double-float "
                   "transforms, float64 pointwise terms); float64 state and stage sums")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the shelf/2d/serving sections after the headline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--only-config", choices=["solitary_1d", "shelf_1d", "bump_2d", "pcg2d_batch",
                                              "generic_sizes", "serving", "robustness",
                                              "manufactured"],
                    help="run only this extra configuration and print its result as one JSON "
                         "line (for profiling one workload; not the headline)")
    ap.add_argument("--batch2d", type=int, default=16,
                    help="instances of the pcg2d_batch configuration")
    ap.add_argument("--serving-requests", type=int, default=240,
                    help="requests of the serving stream (2000: the whole workload)")
    ap.add_argument("--n2d", type=int, default=512, choices=[128, 256, 512, 1024],
                    help="grid side of the bump_2d configuration")
    ap.add_argument("--shelf-steps", type=int, default=2000,
                    help="steps per run of the shelf_1d configuration (2000: the whole run)")
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


def reduce_ranks(t_ms, points, distributed):
    """Whole-job timing over ranks: the slowest rank's time and the sum of the points every
    rank advanced (each rank owns its own instances; no data crosses ranks)."""
    if not distributed:
        return float(t_ms), float(points)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pts = torch.tensor([float(points)], dtype=torch.float64)
    dist.all_reduce(pts, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(pts[0])


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


def _oracle_worker_init():
    # one thread per process: the pool's size is the core count it uses
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    import numpy  # noqa: F401
    from oracle import sgn_oracle  # noqa: F401


def _oracle_step(task):
    """One oracle RK4 step of one instance (a pool task); returns its points."""
    from oracle import sgn_oracle as O
    n, L, g, dt, h, eta, u = task
    st = O.init_state(eta, u, h, O.make_grid(1, n, L, g))
    O.rk4_step(st, dt, RTOL)
    return n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on every host core: a spawn-started process pool (safe after CUDA use),
    one instance's RK4 step per task over a size-stratified sample of the ensemble (six
    tasks per core, largest first, so that the cores finish together)."""

    def __init__(self, ens, workers):
        import multiprocessing as mp
        self.workers = workers
        order = sorted(range(len(ens)), key=lambda i: ens[i].n)
        pick = order[:: max(1, len(order) // (6 * workers))][: 6 * workers]
        pick.sort(key=lambda i: -ens[i].n)        # largest first: the pool balances the rest
        self.tasks = [(c.n, c.L, c.g, c.dt, c.h, c.eta, c.u) for c in (ens[i] for i in pick)]
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init)
        self.pool.map(abs, range(workers), chunksize=1)        # every worker started

    def run(self):
        t0 = time.perf_counter()
        pts = sum(self.pool.map(_oracle_step, self.tasks, chunksize=1))
        return pts, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def reference_arm(args):
    from paper_2506_16045_gb300 import inputs as I
    ens = I.ensemble_1d(count=args.count, seed=2506)
    workers = host_cores()
    pool = OraclePool(ens, workers)
    vals = []
    for _ in range(args.warmup):
        pool.run()
    for _ in range(args.steps):
        vals.append(pool.run())
    pool.close()
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
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{len(pool.tasks)} size-stratified instances x 1 RK4 step "
                                   f"per timed step, one process per core, {pts} "
                                   f"instance-points over {args.steps} steps"},
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

    def autotune(self):
        """Kernel forms (one CTA or a two-CTA cluster per instance, for the solve and the
        right-hand side separately) of the n = 4096 and 8192 classes, timed on RK4 steps of
        this ensemble; the state is restored."""
        self.tune_ms = self.st.autotune(self.dts, rtol=RTOL, maxit=4000,
                                        prec=self.sgn.PREC_MIXED)
        self.forms = {str(1 << l2): dict(zip(("solve", "rhs"), self.lay.forms(l2)))
                      for l2 in (12, 13)}

    def step(self, prec, n=1):
        self.st.rk4(self.dts, n, rtol=RTOL, maxit=4000, prec=prec)

    def launches_per_step(self):
        c = len(self.classes)
        # per RK4 step: 4 right-hand sides and 4 solves per size class, 5 stage combinations,
        # the first stage's starting point, 4 counter updates and the time update (the field
        # copies are memcpy nodes, not kernels)
        return 4 * c + 4 * c + 5 + 1 + 4 + 1


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
    E.autotune()
    ctx.profile(True)         # on for the warm-up too, so the timed steps replay one graph
    for _ in range(args.warmup):
        E.step(sgn.PREC_MIXED)
    torch.cuda.synchronize()
    ctx.profile_read()        # discard the warm-up's launch-group timings
    s0 = E.st.stats()
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
    t_ms, total_points = reduce_ranks(t_ms, E.points, pg is not None)
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

    # ---- the configuration's whole 200-step run: mixed against batched float64 at the end
    E.reset()
    E.step(sgn.PREC_MIXED, FULL_STEPS)
    zm, um = E.eta.cpu().numpy() - E.h.cpu().numpy(), E.u.cpu().numpy()
    E.reset()
    E.step(sgn.PREC_FP64, FULL_STEPS)
    z6, u6 = E.eta.cpu().numpy() - E.h.cpu().numpy(), E.u.cpu().numpy()
    err_full = {"steps": FULL_STEPS, "rel_l2_zeta_vs_fp64": rel(zm, z6),
                "rel_l2_u_vs_fp64": rel(um, u6)}

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

    # ---- end to end through host buffers: the state lives on the host; every step uploads
    # (eta, U, u), steps, and downloads the new (eta, U, u)
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

    def e2e_step():
        E.eta.copy_(h_eta, non_blocking=True)
        E.U.copy_(h_U, non_blocking=True)
        E.u.copy_(h_u, non_blocking=True)
        E.step(sgn.PREC_MIXED)
        h_eta.copy_(E.eta, non_blocking=True)
        h_U.copy_(E.U, non_blocking=True)
        h_u.copy_(E.u, non_blocking=True)

    # untimed warm-up: the steps above ran with profiling on, which is part of the step
    # graph's key, so the library captures its graph again here (as any run does once)
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(ke):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / ke

    # ---- CPU oracle on a bounded sample (rank 0, N = 1) and its agreement after 1 step
    cpu = None
    oracle_err = None
    if rank == 0 and world == 1:
        pts, t_cpu, res = oracle_sample(ens, args.cpu_seconds)
        workers = host_cores()
        pool = OraclePool(ens, workers)
        ppts, pt = pool.run()
        pool.close()
        cpu = {"value": ppts / pt, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{len(pool.tasks)} size-stratified instances x 1 RK4 step ({ppts} "
                         f"points), one process per core, numpy float64, {pt:.1f} s",
               "value_1core": pts / t_cpu,
               "sample_1core": f"{len(res)} instances x 1 RK4 step ({pts} points), "
                               f"{t_cpu:.1f} s"}
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
    # mixed path: the high-precision part runs in double-float, DF_COST float32 operations per
    # nominal flop; achieved is in float32-operation TFLOP/s
    f32 = s1["flops32"] - s0["flops32"]
    fhi = s1["flops64"] - s0["flops64"]
    pcg_s = prof["pcg_ms"] * 1e-3
    achieved = (f32 + DF_COST * fhi) / pcg_s / 1e12
    nominal = (f32 + fhi) / pcg_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
            "frac": achieved * 1e12 / FP32_PEAK, "traffic": None,
            "kernel": "k_pcg1d<float,...,mixed> (one launch per size class per solve)",
            "note": "float32-operation rate: float32 algorithmic flops plus double-float flops "
                    f"x {DF_COST}; peak = 152 SMs x 128 FMA lanes x 2 x 2.07 GHz (derived)",
            "frac_nominal": nominal * 1e12 / FP32_PEAK,
            "achieved_nominal": nominal,
            "note_nominal": "nominal flops (a double-float flop counted once) over the same "
                            "time: the method's work without the cost model of double-float",
            "peak_fp32_probe": FP32_PROBE_TFLOPS,
            "frac_of_probe": achieved / FP32_PROBE_TFLOPS,
            "flops32": f32, "flops_df": fhi,
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
                   "precision": PRECISION_MIXED,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas",
                   "autotuned_ctas_per_instance": E.forms},
        "e2e": {"value": total_points / (e2e_ms * 1e-3) if world == 1 else None, "unit": UNIT,
                "h2d_bytes_per_step": 3 * 8 * P, "d2h_bytes_per_step": 3 * 8 * P},
        "gpu_launches": E.launches_per_step() * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "cpu_baseline": cpu,
        "accuracy": {"rel_l2_eta_vs_fp64": err_eta, "rel_l2_u_vs_fp64": err_u,
                     "rel_l2_zeta_vs_fp64": err_zeta, "steps_compared": nref,
                     "rel_l2_vs_oracle_sample_1step": oracle_err,
                     "whole_run": err_full},
        "batched_fp64": {"value": total_points / (fp64_ms * 1e-3), "unit": UNIT},
        "plain_fp64": plain,
        "step_latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1,
                                                                     int(0.99 * len(srt)))]},
        "solver": {"solves": s1["solves"] - s0["solves"],
                   "iterations": s1["iterations"] - s0["iterations"],
                   "refinements": s1["refinements"] - s0["refinements"],
                   "max_iters": s1["max_iters"], "status": s1["status"]},
    }
    if rank == 0 and world == 1 and not args.no_extra:
        E.st.close()
        extra = {}
        for name, fn in (("solitary_1d", bench_solitary), ("shelf_1d", bench_shelf),
                         ("bump_2d", bench_2d), ("pcg2d_batch", bench_pcg2d),
                         ("generic_sizes", bench_generic),
                         ("serving", bench_serving), ("robustness", bench_robustness),
                         ("manufactured", bench_manufactured)):
            try:
                extra[name] = fn(sgn, ctx, torch)
            except Exception as exc:                          # reported, never silent
                extra[name] = {"error": repr(exc)}
        line["configs"] = extra
        pc = extra.get("pcg2d_batch", {})
        if "persistent_kernel" in pc:
            pk = pc["persistent_kernel"]
            peak, src = hbm_peak()
            tr = PCG2D_TRAFFIC_BYTES
            line["roofline_pcg2d"] = {
                "bound": "hbm", "achieved": pk["algorithmic_GBs"], "peak": peak, "unit": "GB/s",
                "frac": pk["algorithmic_GBs"] / peak, "peak_source": src,
                "traffic": tr,
                "traffic_GBs": tr / (pk["ms_per_launch"] * 1e-3) / 1e9 if tr else None,
                "kernel": "k2_pcg_persist (one persistent launch per float32 inner solve)",
                "workload": pc["workload"],
                "note": "achieved = 60 B per point per inner iteration (eta, grad h read; x, r, p "
                        "of two components read and written, float32) x iterations per launch / "
                        "launch time from CUDA events around each launch"}
        print(json.dumps(line))
        return
    if rank == 0:
        print(json.dumps(line))
    E.st.close()


def bench_solitary(sgn, ctx, torch, steps=500):
    """Flat-bottom solitary wave (L = 100, n = 256, a = 0.2 at x = 25, g = 9.81), float64 RK4
    with PCG at rtol 1e-12, dt = 0.01, the whole 500-step run; the same run in mixed precision
    beside it.  Timed with CUDA events from the initial state after a short untimed run of the
    same kind; the error against the closed-form translate at t = 5 (which carries the
    periodic-image tail, ~1e-7 at L = 100) and the mass drift."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    c = I.solitary_case()
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g)])
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    x = I.grid_1d(c.n, c.L)
    ee, ue = I.solitary_wave_1d(x, c.L, 1.0, 0.2, 25.0, c.g, t=steps * c.dt)
    out = {}
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        for k in (5, steps):
            eta, u, h = dev(c.eta), dev(c.u), dev(c.h)
            U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
            st = sgn.State(lay, eta, U, u, h, gh)
            st.init()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st.rk4(c.dt, k, rtol=1e-12, maxit=2000, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            stats = st.stats()
            st.close()
        out[prec] = (sec, eta.cpu().numpy(), u.cpu().numpy(), stats)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    t6, e6, u6, s6 = out[sgn.PREC_FP64]
    tm, em, um, _ = out[sgn.PREC_MIXED]
    m0 = float(np.sum(c.eta - c.h))
    return {"workload": "solitary_1d: flat-bottom solitary wave L=100, n=256, a=0.2, g=9.81, "
                        f"float64 RK4 + PCG rtol 1e-12, dt 0.01, {steps} steps",
            "steps": steps, "value": c.n * steps / t6, "unit": UNIT, "dtype": "f64",
            "seconds": round(t6, 4), "ms_per_step": 1e3 * t6 / steps,
            "mixed_value": c.n * steps / tm,
            "rel_linf_eta_vs_closed_form": float(np.abs(e6 - ee).max() / np.abs(ee - 1.0).max()),
            "rel_l2_u_vs_closed_form": rel(u6, ue),
            "rel_l2_eta_mixed_vs_fp64": rel(em, e6), "rel_l2_u_mixed_vs_fp64": rel(um, u6),
            "mass_drift_rel": abs(float(np.sum(e6 - c.h)) - m0) / abs(m0),
            "iterations_per_solve": s6["iterations"] / max(1, s6["solves"]),
            "status": s6["status"]}


def bench_pcg2d(sgn, ctx, torch, B=16, n=512, L=80.0, seed=2024, reps=3, radix=8):
    """Batched 2d constraint solves: B instances of the bump workload's size (n^2, L = 80) on
    one grid, each with its own Gaussian bump (height U[0.1, 0.6], radius U[1, 5], centre
    U[0.3L, 0.7L]^2) and wave, right-hand side b = G u* for a smooth u* (formed on the GPU by
    sgn_apply_operator), mixed precision to rtol 1e-10.  The persistent inner-solve kernel is
    timed with CUDA events around each launch (sgn_profile_inner2d); its algorithmic traffic
    is 60 bytes per point per inner iteration (eta and grad h read, x, r, p of two
    components read and written, float32)."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    X, Y = I.grid_2d(n, n, L, L)
    etas, hs, us = [], [], []
    for _ in range(B):
        h = I.gaussian_bump_2d(X, Y, L, L, rng.uniform(0.1, 0.6), rng.uniform(1.0, 5.0),
                               rng.uniform(0.3, 0.7) * L, rng.uniform(0.3, 0.7) * L)
        etas.append(h + rng.uniform(0.05, 0.3) * np.exp(np.cos(2 * np.pi * X / L
                                                                - rng.uniform(0, 6)) - 1))
        hs.append(h)
        k = int(rng.integers(1, 4))
        us.append(np.stack([0.3 * np.sin(2 * np.pi * k * X / L) * np.cos(4 * np.pi * Y / L),
                            0.2 * np.cos(2 * np.pi * X / L) + 0.1 * np.sin(2 * np.pi * k * Y / L)]))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                    device="cuda")
    pack_v = lambda vs: np.concatenate([v[0].ravel() for v in vs] + [v[1].ravel() for v in vs])
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, L, ny=n, Ly=L, g=9.81)] * B)
    lay.set_radix2d(radix)
    eta = dev(np.concatenate([e.ravel() for e in etas]))
    gh = torch.zeros(2 * B * n * n, dtype=torch.float64, device="cuda")
    sgn.spectral_grad(lay, dev(np.concatenate([h.ravel() for h in hs])), gh)
    ustar = dev(pack_v(us))
    b = torch.zeros_like(ustar)
    sgn.apply_operator(lay, eta, gh, ustar, b)
    x = torch.zeros_like(b)
    info = sgn.pcg(lay, eta, gh, b, x, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    ts = []
    for _ in range(reps):
        x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sgn.pcg(lay, eta, gh, b, x, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED, info=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    err = float(torch.linalg.norm(x - ustar) / torch.linalg.norm(ustar))
    lay.profile_inner2d(True)
    for _ in range(reps):
        x.zero_()
        sgn.pcg(lay, eta, gh, b, x, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED, info=False)
    ms, launches, iters = lay.profile_inner2d(False)
    lay.close()
    per_launch_s = ms * 1e-3 / launches
    alg_bytes = 60.0 * n * n * iters / launches        # per launch
    return {"workload": f"pcg2d_batch: {B} instances of {n}^2 (L = {L:g}) on one grid, Gaussian "
                        "bumps, b = G u*, mixed precision, rtol 1e-10",
            "instances": B, "n": n, "max_radix": radix, "solve_ms": min(ts),
            "value": B * n * n / (min(ts) * 1e-3), "unit": "grid-point-solves/s",
            "rel_l2_vs_known_solution": err,
            "inner_iterations_per_instance": [i["iters"] for i in info],
            "refinements_per_instance": [i["refinements"] for i in info],
            "persistent_kernel": {"launches": launches, "ms_per_launch": 1e3 * per_launch_s,
                                  "inner_iterations_per_launch": iters / launches,
                                  "algorithmic_bytes_per_launch": alg_bytes,
                                  "algorithmic_GBs": alg_bytes / per_launch_s / 1e9}}


def bench_2d(sgn, ctx, torch, steps=300, n=512):
    """2d plane solitary wave over a Gaussian bump (80 x 80 at n^2, 512^2 by default; dt 0.02
    at 512^2, scaled with the grid spacing), RK4 over the whole run (300 steps to t = 6 at
    512^2, where the wave has reached the bump), mixed and float64 at rtol 1e-10; the mixed
    run's error against the float64 run at the end, and the mass drift of each."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    c = I.bump2d_case(n=n, L=80.0, a=0.2, x0=20.0, H=0.5, R=3.0, dt=0.02 * 512 / n)
    n = c["n"]
    steps = steps * n // 512
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, c["L"], g=c["g"], ny=n, Ly=c["L"])])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                    device="cuda")
    zeta0 = c["eta"] - c["h"]
    out = {}
    for prec in (sgn.PREC_MIXED, sgn.PREC_FP64):
        for k in (2, steps):                       # a short untimed run, then the whole run
            eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
            U = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
            gh = torch.zeros_like(U)
            st = sgn.State(lay, eta, U, u, h, gh)
            st.init()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st.rk4(c["dt"], k, rtol=1e-10, maxit=4000, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            stats = st.stats()
            st.close()
        out[prec] = (sec, eta.cpu().numpy().reshape(n, n), u.cpu().numpy(), stats)
    tm, em, um, sm = out[sgn.PREC_MIXED]
    t6, e6, u6, _ = out[sgn.PREC_FP64]
    # where a mixed step's time goes: 20 more steps with the library's launch-group events on
    # (the solves and the right-hand sides), after the timed runs
    eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
    U = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    st = sgn.State(lay, eta, U, u, h, torch.zeros_like(U))
    st.init()
    st.rk4(c["dt"], 2, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st.rk4(c["dt"], 20, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    e1.record()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    st.close()
    seg_ms = e0.elapsed_time(e1)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    mass = lambda e: float(np.sum(e - c["h"]))
    m0 = float(np.sum(zeta0))
    return {"workload": f"2d bump 80x80 at {n}^2, RK4 dt {c['dt']:g}, {steps} steps to "
                        f"t = {steps * c['dt']:g}, rtol 1e-10", "steps": steps,
            "value": n * n * steps / tm, "unit": UNIT, "fp64_value": n * n * steps / t6,
            "seconds_mixed": round(tm, 3), "seconds_fp64": round(t6, 3),
            "rel_l2_zeta_vs_fp64": rel(em - c["h"], e6 - c["h"]),
            "rel_l2_u_vs_fp64": rel(um, u6),
            "mass_drift_rel": {"mixed": abs(mass(em) - m0) / abs(m0),
                               "fp64": abs(mass(e6) - m0) / abs(m0)},
            "max_zeta": float(np.abs(em - c["h"]).max()),
            "iterations_per_solve": sm["iterations"] / max(1, sm["solves"]), "status": sm["status"],
            "mixed_step_split": {"steps": 20, "ms_per_step": seg_ms / 20,
                                 "solve_ms_per_step": prof["pcg_ms"] / 20,
                                 "rhs_ms_per_step": prof["rhs_ms"] / 20,
                                 "solve_share": prof["pcg_ms"] / seg_ms,
                                 "rhs_share": prof["rhs_ms"] / seg_ms,
                                 "note": "CUDA events of the library's profiling hooks around "
                                         "each solve and each right-hand side"}}


def bench_generic(sgn, ctx, torch, count=128, steps=20):
    """Sizes that are not powers of two on the generic kernels: a 1d ensemble with n drawn
    from {768, 1536, 3072, 6144} (RK4, mixed, rtol 1e-10) against the same-seed ensemble at
    the power-of-two sizes {512, 1024, 2048, 4096}, and a 2d bump at 384 x 240 (RK4, mixed)
    against 512 x 256."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    out = {}
    for name, sizes in (("generic_1d", [768, 1536, 3072, 6144]),
                        ("pow2_1d", [512, 1024, 2048, 4096])):
        ens = I.ensemble_1d(count=count, seed=2507, sizes=sizes)
        E = Ensemble(sgn, ctx, ens, torch)
        E.reset()
        E.step(sgn.PREC_MIXED, 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        E.step(sgn.PREC_MIXED, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stt = E.st.stats()
        out[name] = {"sizes": sizes, "instances": count, "points": E.points,
                     "ms_per_step": ms / steps, "value": E.points * steps / (ms * 1e-3),
                     "unit": UNIT, "status": stt["status"]}
        E.st.close()
        E.lay.close()
    for name, (nx, ny) in (("generic_2d", (384, 240)), ("pow2_2d", (512, 256))):
        Lx, Ly = 80.0, 50.0
        X, Y = I.grid_2d(nx, ny, Lx, Ly)
        h = I.gaussian_bump_2d(X, Y, Lx, Ly, 0.4, 3.0, Lx / 2, Ly / 2)
        eta, u = I.solitary_wave_2d(X, Y, Lx, Ly, 1.0, 0.2, 0.25 * Lx, 9.81)
        eta = h + (eta - 1.0)
        dt = 0.25 * (Lx / nx) / np.sqrt(9.81 * 1.2)
        lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, g=9.81, ny=ny, Ly=Ly)])
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                        device="cuda")
        E_, u_, h_ = dev(eta), dev(u), dev(h)
        U_ = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        st = sgn.State(lay, E_, U_, u_, h_, torch.zeros_like(U_))
        st.init()
        st.rk4(dt, 2, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.rk4(dt, 10, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stt = st.stats()
        out[name] = {"grid": f"{nx}x{ny}", "ms_per_step": ms / 10,
                     "value": nx * ny * 10 / (ms * 1e-3), "unit": UNIT,
                     "iterations_per_solve": stt["iterations"] / max(1, stt["solves"]),
                     "status": stt["status"]}
        st.close()
        lay.close()
    out["workload"] = ("generic sizes: 1d ensemble of 128 shelf instances, n from {768, 1536, "
                       "3072, 6144}, RK4 mixed rtol 1e-10, 20 steps; 2d bump at 384x240, RK4 "
                       "mixed, 10 steps; each beside its power-of-two neighbour")
    return out


def bench_shelf(sgn, ctx, torch, steps=2000):
    """1d shelf (N = 4096, L = 200, a = 0.3, ramp of width 5 at x = 60), whole 2000-step runs:
    AB4 with PCG (float64, and mixed refined to the same rtol 1e-12) against the linearly
    implicit SBDF2 step (float64 and mixed), each at its own stable step (AB4 dt 0.004, SBDF2
    dt 0.002), SBDF2 with 2/3-rule dealiasing over 4000 steps to t = 8, which it reaches
    only with dealiasing, and RK4 on the constraint and on the non-constraint form (mixed,
    dt 0.004).  Each run is timed with CUDA events from its initial state, start-up steps
    included, after a short untimed run of the same kind."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    c = I.shelf_case()
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g)])
    variants = (("ab4_fp64", "ab4", sgn.PREC_FP64, 1e-12),
                ("ab4_mixed", "ab4", sgn.PREC_MIXED, 1e-12),
                ("sbdf2_fp64", "sbdf2", sgn.PREC_FP64, 1e-12),
                ("sbdf2_mixed", "sbdf2", sgn.PREC_MIXED, 1e-12),
                ("sbdf2_mixed_dealiased_to_t8", "sbdf2", sgn.PREC_MIXED, 1e-12),
                ("rk4_mixed", "rk4", sgn.PREC_MIXED, 1e-12),
                ("rk4_nc_mixed", "rk4_nc", sgn.PREC_MIXED, 1e-12))
    res, final = {}, {}
    for name, scheme, prec, rtol in variants:
        dealias = "dealiased" in name
        dt = I.SHELF_DT.get(scheme, I.SHELF_DT["ab4"])
        nsteps = 2 * steps if dealias else steps          # the dealiased SBDF2 run goes to t = 8
        for k in (8, nsteps):
            eta, u, h = (torch.as_tensor(a, dtype=torch.float64, device="cuda")
                         for a in (c.eta, c.u, c.h))
            U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
            st = sgn.State(lay, eta, U, u, h, gh)
            st.init()
            st.set_dealias(dealias)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            if scheme == "sbdf2":
                st.linimp(dt, k, rtol=rtol, maxit=4000, prec=prec)
            elif scheme == "rk4":
                st.rk4(dt, k, rtol=rtol, maxit=4000, prec=prec)
            elif scheme == "rk4_nc":
                st.rk4_nc(dt, k, rtol=rtol, maxit=4000, prec=prec)
            else:
                st.abk(4, dt, k, rtol=rtol, maxit=4000, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            stats = st.stats()
            st.close()
        final[name] = (eta.cpu().numpy() - c.h, u.cpu().numpy())
        res[name] = {"value": c.n * nsteps / sec, "seconds": round(sec, 4), "dt": dt,
                     "steps": nsteps, "t_final": nsteps * dt,
                     "simulated_time_per_s": nsteps * dt / sec,
                     "status": stats["status"],
                     "iterations_per_solve": stats["iterations"] / max(1, stats["solves"]),
                     "max_zeta": float(np.abs(final[name][0]).max())}
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for s_ in ("ab4", "sbdf2"):
        (zm, um), (z6, u6) = final[s_ + "_mixed"], final[s_ + "_fp64"]
        res[s_ + "_mixed"]["rel_l2_zeta_vs_fp64"] = rel(zm, z6)
        res[s_ + "_mixed"]["rel_l2_u_vs_fp64"] = rel(um, u6)
    # the constraint and non-constraint RK4 runs differ by their time discretisations only
    (zc, uc), (zn, un) = final["rk4_mixed"], final["rk4_nc_mixed"]
    res["rk4_nc_mixed"]["rel_l2_zeta_vs_rk4"] = rel(zn, zc)
    res["rk4_nc_mixed"]["rel_l2_u_vs_rk4"] = rel(un, uc)
    return {"workload": f"1d shelf N=4096 L=200, {steps} steps per run (AB4 and RK4 dt 0.004 "
                        f"to t = {steps * 0.004:g}; SBDF2 dt 0.002 to t = {steps * 0.002:g}; "
                        f"dealiased SBDF2 dt 0.002 to t = {2 * steps * 0.002:g})",
            "unit": UNIT, **res}


def bench_robustness(sgn, ctx, torch, reps=5):
    """The PCG robustness suite of §6.2-§6.3 on the GPU: solve clock time against n for
    Eq:Testproblem (eta0 = h0 = 1, rtol 1e-12; the paper's clock-time-versus-n figure),
    iterations over the eta0 / h0 sweeps, optimal against replacement coefficients on the
    square-wave depth, and the 2d elliptical bump at three aspect ratios."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                    device="cuda")

    def grad_dev(lay, h, comps):
        gh = torch.zeros(comps * h.size, dtype=torch.float64, device="cuda")
        sgn.spectral_grad(lay, dev(h), gh)
        return gh

    def timed(lay, eta, gh, b, npts, rtol, prec, P=None):
        x = torch.zeros(npts, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, eta, gh, b, x, rtol=rtol, maxit=20000, prec=prec, P=P)[0]
        ts = []
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sgn.pcg(lay, eta, gh, b, x, rtol=rtol, maxit=20000, prec=prec, P=P)
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)) * 1e3, info

    clock = []
    for k in range(5, 15):
        n = 2 ** k
        _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
        gh = grad_dev(lay, h, 1)
        row = {"n": n}
        for name, prec in (("fp64", sgn.PREC_FP64), ("mixed", sgn.PREC_MIXED)):
            ms, info = timed(lay, dev(eta), gh, dev(b), n, 1e-12 if name == "fp64" else 1e-11,
                             prec)
            row[f"ms_{name}"] = round(ms, 4)
            row[f"iters_{name}"] = info["iters"]
            row[f"ns_per_nlog2n_{name}"] = round(1e6 * ms / (n * k), 3)
        lay.close()
        clock.append(row)
    sweep = []
    n = 4096
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    for eta0, hvar in ((0.5, 1.0), (1.0, 1.0), (4.0, 1.0), (16.0, 1.0), (1.0, 0.5), (1.0, 2.0),
                       (1.0, 4.0)):
        _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
        gh = grad_dev(lay, h, 1)
        P = sgn.precond_coeffs(lay, dev(eta), gh)
        ms, info = timed(lay, dev(eta), gh, dev(b), n, 1e-12, sgn.PREC_FP64)
        sweep.append({"eta0": eta0, "h0": hvar, "kappa_ub": round(P[0]["kappa_ub"], 1),
                      "iters": info["iters"], "ms": round(ms, 3)})
    square = {}
    lay512 = sgn.Layout(ctx, [sgn.Grid(1, 512, 1.0)])
    for eta0 in (0.25, 5.0):
        _, h, eta, b = I.squarewave_1d(512, eta0)
        gh = grad_dev(lay512, h, 1)
        for name, kind in (("opt", sgn.COEF_OPT), ("replacement", sgn.COEF_REPLACEMENT)):
            P = sgn.precond_coeffs(lay512, dev(eta), gh, kind=kind)
            x = torch.zeros(512, dtype=torch.float64, device="cuda")
            info = sgn.pcg(lay512, dev(eta), gh, dev(b), x, rtol=1e-10, maxit=5000, P=P)[0]
            square[f"eta0={eta0} {name}"] = {"sigma": round(P[0]["sigma"], 5),
                                             "iters": info["iters"]}
    bump = []
    n = 256
    lay2 = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    for a, bb in ((1.0, 1.0), (1.0, 20.0), (1.0, 40.0)):
        _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, bb)
        gh = grad_dev(lay2, h, 2)
        P = sgn.precond_coeffs(lay2, dev(eta), gh)
        ms, info = timed(lay2, dev(eta), gh, dev(rhs), 2 * n * n, 1e-10, sgn.PREC_FP64)
        msm, infom = timed(lay2, dev(eta), gh, dev(rhs), 2 * n * n, 1e-10, sgn.PREC_MIXED)
        bump.append({"a": a, "b": bb, "n": f"{n}^2", "kappa_ub": round(P[0]["kappa_ub"], 1),
                     "iters_fp64": info["iters"], "ms_fp64": round(ms, 3),
                     "iters_mixed": infom["iters"], "ms_mixed": round(msm, 3)})
    # the GMRES option against PCG on the same problems (float64, rtol 1e-10 in the A^{-1}
    # measure for both)
    def timed_gmres(lay, eta, gh, b, npts, restart=30):
        x = torch.zeros(npts, dtype=torch.float64, device="cuda")
        info = sgn.gmres(lay, eta, gh, b, x, rtol=1e-10, restart=restart, maxit=20000)[0]
        ts = []
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sgn.gmres(lay, eta, gh, b, x, rtol=1e-10, restart=restart, maxit=20000)
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)) * 1e3, info

    gmres = []
    for k in (10, 13, 14):
        n = 2 ** k
        _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
        gh = grad_dev(lay, h, 1)
        msg, ig = timed_gmres(lay, dev(eta), gh, dev(b), n)
        msp, ip = timed(lay, dev(eta), gh, dev(b), n, 1e-10, sgn.PREC_FP64)
        gmres.append({"case": f"Eq:Testproblem n={n}", "gmres30_ms": round(msg, 3),
                      "gmres30_steps": ig["iters"], "gmres30_cycles": ig["cycles"],
                      "pcg_fp64_ms": round(msp, 3), "pcg_iters": ip["iters"]})
        lay.close()
    for a, bb in ((1.0, 1.0), (1.0, 20.0)):
        _, _, h, eta, rhs = I.elliptical_bump_2d(256, a, bb)
        gh = grad_dev(lay2, h, 2)
        msg, ig = timed_gmres(lay2, dev(eta), gh, dev(rhs), 2 * 256 * 256)
        msp, ip = timed(lay2, dev(eta), gh, dev(rhs), 2 * 256 * 256, 1e-10, sgn.PREC_FP64)
        gmres.append({"case": f"elliptical bump ({a:g},{bb:g}) 256^2", "gmres30_ms": round(msg, 3),
                      "gmres30_steps": ig["iters"], "gmres30_cycles": ig["cycles"],
                      "pcg_fp64_ms": round(msp, 3), "pcg_iters": ip["iters"]})
    return {"workload": "Eq:Testproblem (eta0 = h0 = 1) solve clock time for n = 2^5..2^14 "
                        "(fp64 rtol 1e-12, mixed rtol 1e-11; one instance per call, median of "
                        f"{reps}); eta0 / h0 sweep at n = 4096; square-wave depth, optimal vs "
                        "replacement coefficients at n = 512; 2d elliptical bump at 256^2",
            "clock_vs_n": clock, "sweep_n4096": sweep, "square_wave_n512": square,
            "elliptical_bump_2d": bump, "gmres_vs_pcg": gmres}


def bench_manufactured(sgn, ctx, torch, n=256, t_final=1.0):
    """Test 1 of §6.4: the forced SGN equations with the manufactured solution (h = 2 +
    sin 2 pi x, eta* = 2 + sin 2 pi x sin 10t, u* = cos 2 pi x cos 10t, L = 1, g = 1) at
    n = 256 to t = 1, every scheme at two step sizes (RK4 C = 0.2, 0.1; SBDF2 C = 0.05,
    0.025, dt = C dx; Adams-Bashforth C = 0.1, 0.05, inside its smaller stability region):
    L-infinity error against the closed form and clock time per run."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    spec = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests",
                                       "golden", "manufactured_forcing.json")))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                    device="cuda")
    x = I.grid_1d(n, 1.0)
    pe, pu, om, th = I.series_forcing_1d(spec, x)
    pe, pu = dev(pe), dev(pu)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0, g=1.0)])
    runs = []
    for name, order, Cs in (("rk4", 0, (0.2, 0.1)), ("ab2", 2, (0.1, 0.05)),
                            ("ab3", 3, (0.1, 0.05)), ("ab4", 4, (0.1, 0.05)),
                            ("sbdf2", 0, (0.05, 0.025))):
        for C in Cs:
            dt = C / n
            steps = int(round(t_final / dt))
            c = I.manufactured_case(n)
            eta, u, h = dev(c.eta), dev(c.u), dev(c.h)
            U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
            st = sgn.State(lay, eta, U, u, h, gh)
            st.init()
            st.set_forcing(pe, pu, om, th)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kw = dict(rtol=1e-12, maxit=4000, prec=sgn.PREC_MIXED)
            if name == "rk4":
                st.rk4(dt, steps, **kw)
            elif name == "sbdf2":
                st.linimp(dt, steps, **kw)
            else:
                st.abk(order, dt, steps, **kw)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            _, e1, u1 = I.manufactured_fields_1d(x, steps * dt)
            runs.append({"scheme": name, "dt": dt, "steps": steps, "seconds": round(sec, 4),
                         "err_eta": float(np.abs(eta.cpu().numpy() - e1).max()),
                         "err_u": float(np.abs(u.cpu().numpy() - u1).max()),
                         "status": st.stats()["status"]})
            st.close()
    orders = {}
    for name in ("rk4", "ab2", "ab3", "ab4", "sbdf2"):
        a, b = [r for r in runs if r["scheme"] == name]
        orders[name] = round(math.log2(max(a["err_eta"], a["err_u"]) /
                                       max(b["err_eta"], b["err_u"])), 2)
    return {"workload": f"forced SGN, manufactured solution of §6.4 Test 1, n = {n}, t = 0 to "
                        f"{t_final}, mixed precision (rtol 1e-12), one instance",
            "runs": runs, "observed_order": orders}


def bench_serving(sgn, ctx, torch, nreq=240, rate=200.0, seed=16045, baseline_sample=8):
    """Poisson stream of SGN runs (RK4, 20-200 steps) and constraint solves (half 1d, half
    2d), host inputs.  A solve's right-hand side is b = G u_s for the solitary-wave velocity
    u_s (formed with sgn_apply_operator before the stream starts), so its answer is known."""
    import numpy as np

    from paper_2506_16045_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    reqs, known = [], {}
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                    device="cuda")
    for _ in range(nreq):
        kind = sgn.REQ_RUN if rng.random() < 0.5 else sgn.REQ_SOLVE
        dim = 1 if rng.random() < 0.5 else 2
        H, R = rng.uniform(0.1, 0.6), rng.uniform(1.0, 5.0)
        a = rng.uniform(0.05, 0.3)
        if dim == 1:
            n, L = 2 ** int(rng.integers(10, 15)), 200.0
            x = I.grid_1d(n, L)
            xb = rng.uniform(0.3, 0.7) * L
            h = 1.0 - H * np.exp(-((x - xb) ** 2) / R ** 2)
            eta, u = I.solitary_wave_1d(x, L, 1.0, a, 0.2 * L, 9.81)
            eta = h + (eta - 1.0)
            grid = sgn.Grid(1, n, L)
            pts = n
        else:
            n, L = 2 ** int(rng.integers(7, 11)), 80.0
            X, Y = I.grid_2d(n, n, L, L)
            xb, yb = rng.uniform(0.3, 0.7, 2) * L
            h = I.gaussian_bump_2d(X, Y, L, L, H, R, xb, yb)
            eta, u = I.solitary_wave_2d(X, Y, L, L, 1.0, a, 0.2 * L, 9.81)
            eta = h + (eta - 1.0)
            grid = sgn.Grid(2, n, L, ny=n, Ly=L)
            pts = n * n
        dx = L / n
        dt = 0.25 * dx / np.sqrt(9.81 * (1 + a))
        nsteps = int(rng.integers(20, 201)) if kind == sgn.REQ_RUN else 0
        if kind == sgn.REQ_SOLVE:
            lay = sgn.Layout(ctx, [grid])
            gh = torch.zeros(dim * pts, dtype=torch.float64, device="cuda")
            sgn.spectral_grad(lay, dev(h), gh)
            b = torch.zeros_like(gh)
            sgn.apply_operator(lay, dev(eta), gh, dev(u), b)
            known[len(reqs)] = np.ascontiguousarray(u, dtype=np.float64).ravel()
            u = b.cpu().numpy()
            lay.close()
        reqs.append((kind, grid, eta, u, h, dt, nsteps, pts))
    srv = sgn.Server(ctx)
    gaps = rng.exponential(1.0 / rate, nreq)
    tickets = []
    t_start = time.perf_counter()
    t_next = t_start
    for i, ((kind, grid, eta, u, h, dt, nsteps, pts), gap) in enumerate(zip(reqs, gaps)):
        t_next += gap
        while time.perf_counter() < t_next:
            time.sleep(0.0002)
        st, t = srv.submit(kind, grid, eta, u, h, scheme=sgn.SCHEME_RK4, dt=dt, nsteps=nsteps,
                           rtol=1e-10, prec=sgn.PREC_MIXED, host=True)
        tickets.append((t, kind, pts, nsteps, st, i))
    done = {}
    while len(done) < len(tickets):
        for t, *_ in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        time.sleep(0.001)
    lat = np.array([1e3 * (done[t]["t_done"] - done[t]["t_submit"]) for t, *_ in tickets])
    solve_lat = np.array([1e3 * (done[t]["t_done"] - done[t]["t_submit"])
                          for t, k, *_ in tickets if k == sgn.REQ_SOLVE])
    by_kind = {}
    for name, kk, dd in (("solve_1d", sgn.REQ_SOLVE, 1), ("solve_2d", sgn.REQ_SOLVE, 2),
                         ("run_1d", sgn.REQ_RUN, 1), ("run_2d", sgn.REQ_RUN, 2)):
        v = np.array([1e3 * (done[t]["t_done"] - done[t]["t_submit"])
                      for t, k, p, ns, st, i in tickets if k == kk and reqs[i][1].dim == dd])
        if v.size:
            by_kind[name] = {"n": int(v.size), "p50_ms": float(np.percentile(v, 50)),
                             "p99_ms": float(np.percentile(v, 99))}
    t0 = min(done[t]["t_submit"] for t, *_ in tickets)
    t1 = max(done[t]["t_done"] for t, *_ in tickets)
    work = sum(p * max(k, 1) for t, kind, p, k, *_ in tickets)    # a solve counts one step
    ok = all(done[t]["status"] == 0 for t, *_ in tickets)
    solve_err = 0.0
    for t, kind, p, k, _, i in tickets:
        if kind == sgn.REQ_SOLVE:
            d = 1 if reqs[i][1].dim == 1 else 2
            x = sgn.device_array(done[t]["u"], d * p).cpu().numpy()
            solve_err = max(solve_err, float(np.linalg.norm(x - known[i]) /
                                             np.linalg.norm(known[i])))
    for t, *_ in tickets:
        srv.release(t)
    srv.close()
    # plain sequential float64 on a sample of the same stream, one request per launch group
    import math
    idx = list(range(0, nreq, max(1, nreq // baseline_sample)))[:baseline_sample]
    wsum, tsum = 0, 0.0
    for i in idx:
        kind, grid, eta, u, h, dt, nsteps, pts = reqs[i]
        lay = sgn.Layout(ctx, [grid])
        d = 1 if grid.dim == 1 else 2
        e_, u_, h_ = (torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64,
                                      device="cuda") for a in (eta, u, h))
        U_ = torch.zeros(d * pts, dtype=torch.float64, device="cuda")
        g_ = torch.zeros_like(U_)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        if kind == sgn.REQ_RUN:
            st = sgn.State(lay, e_, U_, u_, h_, g_)
            st.init()
            st.rk4(dt, nsteps, rtol=1e-10, maxit=4000, prec=sgn.PREC_FP64)
            torch.cuda.synchronize()
            st.close()
        else:
            sgn.spectral_grad(lay, h_, g_)
            sgn.pcg(lay, e_, g_, u_, U_, rtol=1e-10, maxit=4000, prec=sgn.PREC_FP64)
        torch.cuda.synchronize()
        tsum += time.perf_counter() - ts
        wsum += pts * max(nsteps, 1)
    return {"workload": f"Poisson {rate:.0f}/s, {nreq} requests (seed {seed}): 50% RK4 runs "
                        "(20-200 steps) / 50% solves of G x = G u_s, 50% 1d n in 2^10..2^14 / "
                        "50% 2d 2^7..2^10 per side, Gaussian bumps, mixed precision, rtol 1e-10",
            "all_ok": ok, "solve_max_rel_err_vs_known": solve_err,
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "solve_p50_ms": float(np.percentile(solve_lat, 50)) if solve_lat.size else None,
            "solve_p99_ms": float(np.percentile(solve_lat, 99)) if solve_lat.size else None,
            "latency_by_kind": by_kind,
            "sample_reason": None if nreq >= 2000 else
            f"{nreq} of the workload's 2000 requests: the 2d runs (up to 1024^2 x 200 RK4 steps) "
            "share one lane, and the whole stream takes minutes; --serving-requests 2000 runs "
            "all of it",
            "throughput": work / (t1 - t0), "unit": UNIT,
            "plain_fp64_sequential": wsum / tsum,
            "plain_sample": f"{len(idx)} requests of the same stream run one at a time"}


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    if args.only_config:
        import torch

        from paper_2506_16045_gb300 import sgn
        ctx = sgn.Context(0)
        fn = {"solitary_1d": bench_solitary,
              "pcg2d_batch": lambda *a: bench_pcg2d(*a, B=args.batch2d, n=args.n2d),
              "shelf_1d": lambda *a: bench_shelf(*a, steps=args.shelf_steps),
              "bump_2d": lambda *a: bench_2d(*a, n=args.n2d),
              "serving": lambda *a: bench_serving(*a, nreq=args.serving_requests),
              "robustness": bench_robustness,
              "generic_sizes": bench_generic,
              "manufactured": bench_manufactured}
        print(json.dumps({args.only_config: fn[args.only_config](sgn, ctx, torch)}))
        ctx.close()
        return
    gpu_arm(args, world, rank, local, pg)


if __name__ == "__main__":
    main()
