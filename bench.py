#!/usr/bin/env python
"""Benchmark of the McMg online solve on one B300 (or N replicas).

A step is one full solve of the workload to true FP64 relative residual 1e-6:
restarted flexible GMRES preconditioned by one McMg V-cycle per iteration
(every row of the hot path: operator, lift, smoothing, restriction,
prolongation, projection, Krylov orthogonalisation, solution update).

Default workload: the largest single-GPU configuration, 256^3 grid, 7-point
stencil, Gaussian-random-field medium (c in [1, 3], correlation 16 cells)
with three spheres of 5x contrast, 8 points per wavelength at c = 1, 10-cell
sponge, 5 levels with 8/16/32/64/64 channels, FGMRES(30), one point source,
with FP32-accurate channel mixing (three TF32 tensor-core products per FP32
product where the kernels exist, FP32 FFMA elsewhere); the same solve with
BF16 channel mixing is reported beside it under "bf16".  Inputs and the setup
are resident on the device before the timed region; each timed solve is
bracketed by CUDA events on its stream and L2 is flushed (a 256 MiB write)
between solves, outside the events.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload: a few FGMRES iterations per step on the same
recipe (on a 4x coarser copy of the grid when the grid has more than 2^18
nodes, scaled by the node ratio, the oracle's cost per iteration being
linear in the nodes), scaled to a full solve by the stored oracle iteration
count or, without one, the GPU's.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s and V-cycles/s to rel. residual 1e-6; p50/p99 solve latency"
# Iteration cap per workload (the restart length is the workload's FGMRES(m)).
MAX_ITERS = {"helm2d_n64_homogeneous": 2000, "helm2d_n64_slmg": 2000, "helm2d_n256_grf": 4000,
             "helm2d_n1024_layers": 20000, "helm3d_n256_grf": 8000, "helm2d_n256_layers": 20000,
             "helm3d_n64_grf": 4000}
# GPU iteration counts of the workloads whose full-size oracle solve is out of
# reach, to scale the oracle's sampled iterations (FP32-accurate mixing; B300)
GPU_ITERS = {"helm3d_n256_grf": 227, "helm2d_n1024_layers": 8690}
# DRAM bytes (read + write) per launch of the dominant launch class, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (workload, precision, level, kind); the profile summaries record the
# command and the scaling.  A key is dropped when its kernel changes.
NCU_TRAFFIC = {("helm3d_n256_grf", "fp32tc", 1, "step"): 1074503936 + 253044736}
FP32_LANES_PER_SM = 128
NUM_SMS = 148


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mcmg", choices=["mcmg", "reference"])
    p.add_argument("--workload", default="helm3d_n256_grf")
    p.add_argument("--precision", default="fp32tc", choices=["native", "fp32", "bf16", "fp32tc"],
                   help="channel-mixing precision ('native': the workload's own)")
    p.add_argument("--no-bf16", action="store_true", help="skip the BF16 comparison solves")
    p.add_argument("--arrival-x", type=float, default=4.0,
                   help="serving_stream: Poisson arrival rate as a multiple of the plain form's "
                        "request rate (above the served/plain ratio to be measured, so that the "
                        "server, not the arrivals, sets the makespan)")
    p.add_argument("--profile-solve", type=int, default=0,
                   help="profiling aid: after setup, one solve of at most this many FGMRES "
                        "iterations inside the NVTX range 'solve' (ncu --nvtx --nvtx-include "
                        "'solve/'), then exit")
    p.add_argument("--profile-launch", default="",
                   help="LEVEL,KIND[,REPS[,SHAPE]]: after setup, run only that launch class "
                        "of the V-cycle (KIND first | step | residual | restrict | prolong; "
                        "restrict is the residual followed by the restriction) once untimed "
                        "and REPS times (default 5) timed, in kernel shape SHAPE (default: "
                        "setup's choice), and exit; for profilers")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-iters", type=int, default=3)
    p.add_argument("--n", type=int, default=0,
                   help="override the grid size (smaller copies of a workload for profiling)")
    p.add_argument("--max-iters", type=int, default=0)
    p.add_argument("--requests", type=int, default=24,
                   help="serving_stream: how many requests of the 256-request stream to serve")
    p.add_argument("--budget-gb", type=float, default=150.0)
    p.add_argument("--shapes", default="",
                   help="JSON [[op0, op1, op2, op3] per level] of CUDA-core kernel shapes to "
                        "use instead of setup's timed choice (the line's kernel_shapes); keeps "
                        "a profiler run on the kernels a plain run chose")
    return p.parse_args()


def replica_total(total, world, device):
    """Whole-job seconds of `world` replicas: every rank passes its own timed
    region, all get the maximum (the job ends with the slowest replica).
    One rank: unchanged.  Ends with a barrier."""
    if world <= 1:
        return total
    import torch
    import torch.distributed as dist
    t = torch.tensor([total], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_rate(units_per_rank, world, total):
    """Units per second of the whole job: what all replicas processed over
    the job's (max-over-ranks) time."""
    return units_per_rank * world / total


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def setup_workload(name, n=0):
    from paper_2606_30495_b300 import inputs as I
    wl = I.workload(name, **({"n": n} if n else {}))
    c = I.medium_for(wl)
    omega = I.omega_for_ppw(c.min(), wl["ppw"], wl["n"])
    w = I.weights_for(wl)
    return wl, c, omega, w


def smooth_bytes(C, first):
    """Algorithmic bytes per node of one smoothing launch (complex64): read e,
    r, a, s and write e (40 C); the first pre-step (e = 0) reads r, s, writes e
    (24 C)."""
    return (24 if first else 40) * C


def smooth_flops(C, d, first):
    """Algorithmic real flops per node of one smoothing launch: complex MACs
    (8 flops each) of the stencil, K_A, K_S and W^(i); the first pre-step
    (e = 0) has only K_S and W^(i)."""
    return 8 * (2 if first else (2 * d + 4)) * C * C


def residual_bytes(C):
    """Residual t = r - A_l(e): read e, r, a, write t (32 C bytes per node)."""
    return 32 * C


def residual_flops(C, d):
    """Residual: complex MACs of the stencil and K_A (8 (2d + 2) C^2)."""
    return 8 * (2 * d + 2) * C * C


def kernel_family(prec_name, C):
    """Which kernel runs a level's smoothing step and residual: 'ts' (tensor
    cores, A operands in tensor memory; BF16 or FP32-accurate mixing, C >= 8)
    or 'cuda' (FP32 on the CUDA cores)."""
    if prec_name in ("bf16", "fp32tc") and C >= 8:
        return "ts"
    return "cuda"


def time_smoothing(h, wl, torch, stream, reps=20):
    """CUDA-event time of every smoothing and residual launch class of one
    V-cycle, through the C ABI on `stream`.  Returns per-family totals
    {family: dict(flops, bytes, s, launches)} and the per-class detail."""
    d = wl["dim"]
    fams = {}
    detail = []
    for l in range(wl["levels"]):
        C = wl["channels"][l]
        shp = tuple(n >> l for n in (wl["n"],) * d) + (C,)
        nodes = math.prod(shp[:-1])
        r = torch.randn(shp, dtype=torch.complex64, device="cuda")
        e = torch.randn(shp, dtype=torch.complex64, device="cuda")
        o = torch.empty_like(e)
        n_full = wl["nu_pre"][l] + wl["nu_post"][l] - (1 if wl["nu_pre"][l] > 0 else 0)
        n_first = 1 if wl["nu_pre"][l] > 0 else 0
        n_res = 1 if l < wl["levels"] - 1 else 0
        fam = kernel_family(wl["precision"], C)
        for kind, count in (("first", n_first), ("step", n_full), ("residual", n_res)):
            if count == 0:
                continue
            if kind == "residual":
                run = lambda: h.residual(l, r, e, o, stream=stream)
                fl, by = residual_flops(C, d) * nodes, residual_bytes(C) * nodes
                kf = fam
            else:
                first = kind == "first"
                run = lambda: h.smooth(l, 0, r, None if first else e, o, stream=stream)
                fl, by = smooth_flops(C, d, first) * nodes, smooth_bytes(C, first) * nodes
                kf = fam
            with torch.cuda.stream(stream):
                for _ in range(3):
                    run()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    run()
                e1.record(stream)
            e1.synchronize()
            per = e0.elapsed_time(e1) / 1e3 / reps
            f = fams.setdefault(kf, dict(flops=0.0, bytes=0.0, s=0.0, launches=0))
            f["flops"] += fl * count
            f["bytes"] += by * count
            f["s"] += per * count
            f["launches"] += count
            detail.append(dict(level=l, C=C, kind=kind, family=kf, count=count, us=per * 1e6,
                               tflops=fl / per / 1e12, gbs=by / per / 1e9))
    return fams, detail


def time_transfers(h, wl, torch, stream, reps=20):
    """CUDA-event time of the restriction and prolongation of every level, as
    the V-cycle runs them (setup's kernel shapes), through the C ABI on
    `stream`: the prolongation alone (mcmg_prolong_add), the restriction as
    residual + restriction less the residual.  Algorithmic bytes: the input
    read once and the output written (and, prolongation, read) once;
    flops: 8 flops per complex MAC over the 3^d taps of every coarse node."""
    d = wl["dim"]
    T3 = 3 ** d
    out = []
    for l in range(wl["levels"] - 1):
        C, Cn = wl["channels"][l], wl["channels"][l + 1]
        shp = tuple(n >> l for n in (wl["n"],) * d)
        cshp = tuple(n >> (l + 1) for n in (wl["n"],) * d)
        nf, nc = math.prod(shp), math.prod(cshp)
        r = torch.randn(shp + (C,), dtype=torch.complex64, device="cuda")
        e = torch.randn(shp + (C,), dtype=torch.complex64, device="cuda")
        t = torch.empty_like(e)
        rc = torch.empty(cshp + (Cn,), dtype=torch.complex64, device="cuda")
        ec = torch.randn(cshp + (Cn,), dtype=torch.complex64, device="cuda")

        def timed(run):
            with torch.cuda.stream(stream):
                for _ in range(3):
                    run()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    run()
                e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps

        t_res = timed(lambda: h.residual(l, r, e, t, stream=stream))
        t_rr = timed(lambda: h.residual_restrict(l, r, e, rc, stream=stream))
        t_p = timed(lambda: h.prolong_add(l, ec, e, stream=stream))
        fl = 8.0 * T3 * C * Cn * nc
        for kind, sec, by, op in (("restrict", max(t_rr - t_res, 1e-9), 8.0 * (C * nf + Cn * nc), 2),
                                  ("prolong", t_p, 8.0 * (Cn * nc + 2 * C * nf), 3)):
            sh = h.kernel_shape(l, op)
            out.append(dict(level=l, C=C, Cn=Cn, kind=kind, shape=sh, us=sec * 1e6,
                            tflops=fl / sec / 1e12, gbs=by / sec / 1e9))
    return out


def sample_size(wl):
    """Grid size of the oracle's sample: the workload's own up to 2^18 nodes,
    else a 4x coarser copy of the same recipe."""
    return wl["n"] if wl["n"] ** wl["dim"] <= (1 << 18) else wl["n"] // 4


def oracle_rate(name, wl, iters_full, sample_iters):
    """The FP64 oracle timed on the host: `sample_iters` FGMRES iterations
    (one V-cycle + Gram-Schmidt each) on the workload's recipe at
    sample_size(wl), scaled by the node ratio to the full grid and by
    iters_full to a full solve (the setup is outside the timing, as on the GPU)."""
    from oracle import mcmg_oracle as O
    from paper_2606_30495_b300 import inputs as I
    ns = sample_size(wl)
    ws = I.workload(name, n=ns)
    for k in ("precision",):
        ws[k] = wl[k]
    c = I.medium_for(ws)
    omega = I.omega_for_ppw(c.min(), ws["ppw"], ns)
    w = I.weights_for(ws)
    q = O.wavenumber_coef(c, omega, ws["sponge"], ws["gamma_max"])
    feats = O.setup(q, w)
    f = I.point_source(c.shape)
    t0 = time.perf_counter()
    O.fgmres(lambda u: O.apply_A(q, u), lambda v: O.vcycle(w, feats, v), f,
             m=sample_iters + 1, tol=1e-300, max_iters=sample_iters)
    dt = time.perf_counter() - t0
    scale = (wl["n"] / ns) ** wl["dim"]
    per_iter = dt / sample_iters * scale
    return dict(per_iter_s=per_iter, solve_s=per_iter * iters_full, wall_s=dt, n_sample=ns,
                scale=scale)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def golden_iters(name):
    path = os.path.join(ROOT, "tests", "golden", "oracle_solves.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if name in d:
            return d[name]["iters"], "oracle"
    return None, None


def profile_launch(args, h, wl, torch, mcmg, ctx):
    """Run one launch class of the V-cycle (level, kind) on random fields of
    that level, REPS times on one stream, and print its mean CUDA-event time."""
    parts = args.profile_launch.split(",")
    level, kind = int(parts[0]), parts[1]
    reps = int(parts[2]) if len(parts) > 2 else 5
    shape = int(parts[3]) if len(parts) > 3 else -1
    op = {"first": mcmg.OP_SMOOTH, "step": mcmg.OP_SMOOTH, "residual": mcmg.OP_RESIDUAL,
          "restrict": mcmg.OP_RESTRICT, "prolong": mcmg.OP_PROLONG}[kind]
    if shape >= 0 and not h.set_kernel_shape(level, op, shape):
        raise SystemExit(f"kernel shape {shape} cannot run {kind} on level {level}")
    C = wl["channels"][level]
    shp = tuple(n >> level for n in (wl["n"],) * wl["dim"]) + (C,)
    r = torch.randn(shp, dtype=torch.complex64, device="cuda")
    e = torch.randn(shp, dtype=torch.complex64, device="cuda")
    o = torch.empty_like(e)
    stream = torch.cuda.Stream()
    if kind in ("restrict", "prolong"):          # the level's transfer (setup's kernel)
        Cn = wl["channels"][level + 1]
        cshp = tuple(n >> (level + 1) for n in (wl["n"],) * wl["dim"]) + (Cn,)
        rc = torch.empty(cshp, dtype=torch.complex64, device="cuda")
        ec = torch.randn(cshp, dtype=torch.complex64, device="cuda")
    run = {"first": lambda: h.smooth(level, 0, r, None, o, stream=stream),
           "step": lambda: h.smooth(level, 0, r, e, o, stream=stream),
           "residual": lambda: h.residual(level, r, e, o, stream=stream),
           "restrict": lambda: h.residual_restrict(level, r, e, rc, stream=stream),
           "prolong": lambda: h.prolong_add(level, ec, e, stream=stream)}[kind]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        run()                                    # untimed: first-call allocations
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
    e1.synchronize()
    print(json.dumps({"profile_launch": {"workload": args.workload, "precision": wl["precision"],
                                         "level": level, "kind": kind, "C": C,
                                         "shape": h.kernel_shape(level, op),
                                         "nodes": math.prod(shp[:-1]), "reps": reps,
                                         "us": e0.elapsed_time(e1) * 1e3 / reps}}))
    h.close()
    ctx.close()


def profile_solve(args, h, c, wl, torch, mcmg, ctx):
    """One warm-up solve of a few iterations, then one of args.profile_solve
    iterations inside the NVTX range 'solve'; prints its CUDA-event time."""
    from paper_2606_30495_b300 import inputs as I
    f = torch.from_numpy(I.point_source(c.shape)).to("cuda", torch.complex128)
    u = torch.zeros(c.shape, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.solve(f, u, tol=wl["tol"], restart_m=wl["restart"], max_iters=4, stream=stream)
        u.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("solve")
    e0.record(stream)
    st, info = h.solve(f, u, tol=wl["tol"], restart_m=wl["restart"], max_iters=args.profile_solve,
                       stream=stream)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_solve": {"workload": args.workload, "precision": wl["precision"],
                                        "iters": info["iters"], "ms": e0.elapsed_time(e1)}}))
    h.close()
    ctx.close()


def config_of(args, wl, restart):
    return {"workload": args.workload, "grid": [wl["n"]] * wl["dim"], "levels": wl["levels"],
            "channels": wl["channels"], "nu_pre": wl["nu_pre"], "nu_post": wl["nu_post"],
            "fgmres_restart": restart, "tol": wl["tol"], "precision": wl["precision"],
            "l2": "flushed between solves (256 MiB write)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2606_30495_b300 import inputs as I
    wl = I.workload(args.workload, **({"n": args.n} if args.n else {}))
    if args.precision != "native":
        wl["precision"] = args.precision
    iters, src = golden_iters(args.workload)
    if iters is None:
        iters, src = GPU_ITERS.get(args.workload), "gpu"
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no iteration count to scale the oracle's sample for {args.workload}"}))
        return
    k = max(1, args.cpu_sample_iters)
    for _ in range(args.warmup):
        oracle_rate(args.workload, wl, iters, 1)
    walls, solves = [], []
    for _ in range(args.steps):
        o = oracle_rate(args.workload, wl, iters, k)
        walls.append(o["wall_s"])
        solves.append(o["solve_s"])
    value = args.steps / sum(solves)
    cores = cpu_cores()
    sample = (f"{k} FGMRES iterations per step of the FP64 numpy oracle on the recipe at "
              f"{o['n_sample']}^{wl['dim']}, scaled by the node ratio {o['scale']:.0f} and to a "
              f"{iters}-iteration solve ({'oracle count' if src == 'oracle' else 'GPU count'})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": dict(config_of(args, wl, wl["restart"]), parallelism=f"replicas{args.gpus}"),
        "value_from": "solves/s extrapolated from the sampled iterations; ms_per_step is the "
                      "wall time of one sampled step",
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def run_serving(args):
    """Serving stream: requests with their own media and 1-8 point sources.

    Plain form: every right-hand side solved one after another with mcmg_solve
    (one right-hand side per call, no batching) on FP32 handles.  Served form:
    BF16 handles set up at each request's arrival and submitted to the
    context's server (admission against the HBM budget, every request on its
    own stream, the V-cycles due in the same round batched across requests
    into one tensor-core launch per level and step).  Arrivals are Poisson at
    --arrival-x times the plain form's request rate (default 4: at 1.5x, an
    earlier setting, the makespan was bounded by the last arrival and no
    ratio above ~1.7 could be observed).
    Reports solves/s (right-hand sides per second of makespan), p50/p99 request
    latency (completion - arrival, setup included) and the speedup."""
    import numpy as np
    import torch

    from paper_2606_30495_b300 import build as B
    B.build()
    from paper_2606_30495_b300 import inputs as I
    from paper_2606_30495_b300 import mcmg
    torch.cuda.set_device(0)
    base = I.serving_weights()
    reqs = I.serving_requests(count=256)[: args.requests]
    data = [I.serving_request_inputs(r, base) for r in reqs]
    nrhs_total = sum(r["nrhs"] for r in reqs)
    max_it = args.max_iters or 20000
    ctx = mcmg.Context(0, hbm_budget_bytes=int(args.budget_gb * 2 ** 30))

    # ---- plain per-request FP32 form (sequential)
    plain_lat, plain_iters = [], []
    t0 = time.perf_counter()
    for r, (c, om, w, f) in zip(reqs, data):
        ts = time.perf_counter()
        h = mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=mcmg.FP32)
        its = 0
        for j in range(r["nrhs"]):
            fd = torch.from_numpy(np.ascontiguousarray(f[j])).cuda()
            u = torch.zeros_like(fd)
            st, info = h.solve(fd, u, tol=1e-6, restart_m=30, max_iters=max_it)
            its = max(its, info["iters"])
        torch.cuda.synchronize()
        plain_lat.append(time.perf_counter() - ts)
        plain_iters.append(its)
        h.close()
    plain_total = time.perf_counter() - t0
    plain_rate = nrhs_total / plain_total
    req_rate = args.arrival_x * len(reqs) / plain_total

    # ---- served form: Poisson arrivals at req_rate
    rng = np.random.Generator(np.random.PCG64(11))
    gaps = rng.exponential(1.0 / req_rate, size=len(reqs))
    arrive = np.cumsum(gaps) - gaps[0]
    handles, bufs, tickets, t_arr = [], [], [], []
    launches0 = mcmg.kernel_launches()
    t0 = time.perf_counter()
    for k, (r, (c, om, w, f)) in enumerate(zip(reqs, data)):
        while time.perf_counter() - t0 < arrive[k]:
            time.sleep(0.0005)
        t_arr.append(time.perf_counter() - t0)
        h = mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=mcmg.BF16)
        fd = torch.from_numpy(f).cuda()
        u = torch.zeros_like(fd)
        torch.cuda.synchronize()
        tickets.append(ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=max_it,
                                  nrhs=r["nrhs"]))
        handles.append(h)
        bufs.append((fd, u))
    done = {}
    while len(done) < len(tickets):
        for k, t in enumerate(tickets):
            if k in done:
                continue
            st, info = ctx.poll(t)
            if st != mcmg.MCMG_PENDING:
                done[k] = (time.perf_counter() - t0, st, info)
        time.sleep(0.0005)
    makespan = max(v[0] for v in done.values())
    launches = mcmg.kernel_launches() - launches0
    cohort_rounds, cohort_members = ctx.batching()
    lat = sorted(done[k][0] - t_arr[k] for k in range(len(reqs)))
    conv = all(done[k][1] == 0 for k in range(len(reqs)))
    served_rate = nrhs_total / makespan
    # true residuals against the FP64 operator (oracle), every right-hand side
    from oracle import mcmg_oracle as O
    worst = 0.0
    for k, (r, (c, om, w, f)) in enumerate(zip(reqs, data)):
        q = O.wavenumber_coef(c, om, 16, 1.0)
        un = bufs[k][1].cpu().numpy()
        for j in range(r["nrhs"]):
            worst = max(worst, float(np.linalg.norm(f[j] - O.apply_A(q, un[j])) / np.linalg.norm(f[j])))
    dev_err = [h.device_error() for h in handles]
    for h in handles:
        h.close()
    ctx.close()
    pct = lambda a, p: a[min(len(a) - 1, int(math.ceil(p * len(a))) - 1)]
    out = {
        "metric": METRIC, "value": served_rate, "unit": "solves/s", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": 1e3 * makespan, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16/f32", "data": "synthetic",
        "config": {"workload": "serving_stream", "requests": len(reqs), "rhs_total": nrhs_total,
                   "grids": sorted({r["n"] for r in reqs}), "arrival_rate_hz": req_rate,
                   "arrival_rate_x_plain": args.arrival_x,
                   "fgmres_restart": 30, "tol": 1e-6},
        "latency_ms": {"p50": 1e3 * pct(lat, 0.5), "p99": 1e3 * pct(lat, 0.99)},
        "plain_fp32": {"solves_per_s": plain_rate, "seconds": plain_total,
                       "latency_ms_p50": 1e3 * sorted(plain_lat)[len(plain_lat) // 2],
                       "iters": plain_iters},
        "speedup_vs_plain": served_rate / plain_rate,
        "served_iters": [done[k][2]["iters"] for k in range(len(reqs))],
        "served_status": [mcmg.STATUS.get(done[k][1], done[k][1]) for k in range(len(reqs))],
        "served_device_error": dev_err,
        "converged": conv, "worst_true_rel_residual": worst, "gpu_launches": int(launches),
        "cross_request_batching": {"cohort_vcycles": cohort_rounds,
                                   "requests_in_cohorts": cohort_members},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving_stream":
        return run_serving(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_2606_30495_b300 import build as B
    B.build()
    from paper_2606_30495_b300 import inputs as I
    from paper_2606_30495_b300 import mcmg

    wl, c, omega, w = setup_workload(args.workload, args.n)
    if args.precision != "native":
        wl["precision"] = args.precision
    sp = dict(restart=wl["restart"], max_iters=args.max_iters or MAX_ITERS[args.workload])
    prec = {"fp32": mcmg.FP32, "bf16": mcmg.BF16, "fp32tc": mcmg.FP32_TC}[wl["precision"]]
    ctx = mcmg.Context(local)
    t0 = time.perf_counter()
    h = mcmg.Handle(ctx, c, omega, wl["sponge"], wl["gamma_max"], w, precision=prec)
    t_setup = time.perf_counter() - t0
    if args.profile_launch:
        return profile_launch(args, h, wl, torch, mcmg, ctx)
    if args.profile_solve:
        return profile_solve(args, h, c, wl, torch, mcmg, ctx)
    if args.shapes:
        for l, ops in enumerate(json.loads(args.shapes)):
            for op, sh in enumerate(ops):
                if not h.set_kernel_shape(l, op, sh):
                    raise SystemExit(f"shape {sh} cannot run op {op} on level {l}")
    kernel_shapes = [[h.kernel_shape(l, op) for op in range(4 if l < wl["levels"] - 1 else 2)]
                     for l in range(wl["levels"])]
    shape = c.shape
    n = int(np.prod(shape))
    f_host = I.point_source(shape)
    f = torch.from_numpy(f_host).to("cuda", torch.complex128)
    u = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def solve():
        with torch.cuda.stream(stream):
            u.zero_()
        return h.solve(f, u, tol=wl["tol"], restart_m=sp["restart"], max_iters=sp["max_iters"],
                       stream=stream)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    clk.start()
    launches0 = mcmg.kernel_launches()
    times, infos = [], []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = solve()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        infos.append((st, info))
    torch.cuda.synchronize()
    launches = mcmg.kernel_launches() - launches0 - 0
    clocks = clk.stop()
    total = replica_total(sum(times), world, "cuda")
    iters = [i["iters"] for _, i in infos]
    res = max(i["rel_residual"] for _, i in infos)
    conv = all(i["converged"] for _, i in infos)
    value = job_rate(args.steps, world, total)

    # final answer checked against the FP64 operator (oracle) on rank 0
    true_res = None
    if rank == 0:
        from oracle import mcmg_oracle as O
        q = O.wavenumber_coef(c, omega, wl["sponge"], wl["gamma_max"])
        un = u.cpu().numpy()
        true_res = float(np.linalg.norm(f_host - O.apply_A(q, un)) / np.linalg.norm(f_host))

    # standalone V-cycle rate (graph replay, steady state)
    r = torch.randn(shape, dtype=torch.complex64, device="cuda")
    e = torch.empty_like(r)
    with torch.cuda.stream(stream):
        for _ in range(5):
            h.vcycle(r, e, stream=stream)
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        nv = 50
        for _ in range(nv):
            h.vcycle(r, e, stream=stream)
        v1.record(stream)
    v1.synchronize()
    vc_s = v0.elapsed_time(v1) / 1e3 / nv

    # the dominant launch class of the smoothing steps and residuals of one V-cycle
    fams, detail = time_smoothing(h, wl, torch, stream)
    pk, pk_src = peaks()
    ffma_peak = mcmg.fp32_ffma_tflops(stream)          # measured live, this GPU, this run
    dom = max(detail, key=lambda x: x["count"] * x["us"])
    t_launch = dom["us"] * 1e-6
    if dom["family"] == "cuda":
        roof = {"bound": "alu", "achieved": dom["tflops"], "peak": ffma_peak, "unit": "TFLOP/s",
                "peak_source": "measured FFMA loop (mcmg_fp32_ffma_tflops), this run",
                "kernel": "CUDA-core FP32 smoothing step / residual"}
    elif dom["family"] in ("ts", "tc") and dom["C"] <= 16:
        roof = {"bound": "hbm", "achieved": dom["gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "peak_source": f"measured copy bandwidth ({pk_src})",
                "kernel": "k_smooth_ts (tcgen05, A operands in tensor memory)"}
    else:
        # a contraction: executed tensor flops against the peak of its own operand type
        tf = wl["precision"] == "fp32tc"
        mult = 3.0 if tf else 1.0
        peak = pk["bf16_tflops"] * (1.1 / 2.25 if tf else 1.0)
        roof = {"bound": "tensor", "achieved": dom["tflops"] * mult, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": (f"measured cuBLAS BF16 burst ({pk_src})"
                                + (" x nominal TF32/BF16 ratio 1.1/2.25" if tf else "")),
                "kernel": "k_smooth_tsb (tcgen05, streamed weights)" + (", 3 TF32 products"
                                                                         if tf else "")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["launch"] = {k: dom[k] for k in ("level", "C", "kind", "count", "us")}
    roof["traffic"] = NCU_TRAFFIC.get((args.workload, wl["precision"], dom["level"], dom["kind"]))
    roof["families"] = {k: dict(v, share=v["s"] / sum(x["s"] for x in fams.values()))
                        for k, v in fams.items()}
    roof["detail"] = detail
    transfers = time_transfers(h, wl, torch, stream)
    t_smooth = sum(x["us"] * x["count"] for x in detail) * 1e-6
    t_xfer = sum(x["us"] for x in transfers) * 1e-6

    # end to end through the C ABI with host buffers (copies inside the call)
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.zeros(shape, dtype=torch.complex128).pin_memory()
    e2e_times = []
    for k in range(max(2, args.steps // 2)):
        u_pin.zero_()
        t1 = time.perf_counter()
        h.solve_host(f_pin, u_pin, tol=wl["tol"], restart_m=sp["restart"],
                     max_iters=sp["max_iters"])
        e2e_times.append(time.perf_counter() - t1)
    e2e_value = job_rate(len(e2e_times), world, replica_total(sum(e2e_times), world, "cuda"))

    # the same solve with BF16 channel mixing (reported beside the headline)
    bf16 = None
    if not args.no_bf16 and prec != mcmg.BF16:
        hb = mcmg.Handle(ctx, c, omega, wl["sponge"], wl["gamma_max"], w, precision=mcmg.BF16)
        bt, bi = [], []
        for k in range(3):
            with torch.cuda.stream(stream):
                u.zero_()
                flush.fill_(k & 0xFF)
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            stb, ib = hb.solve(f, u, tol=wl["tol"], restart_m=sp["restart"],
                               max_iters=sp["max_iters"], stream=stream)
            b1.record(stream)
            b1.synchronize()
            if k > 0:                                   # the first one warms up
                bt.append(b0.elapsed_time(b1) / 1e3)
                bi.append(ib)
        bf16 = {"value": len(bt) / sum(bt), "unit": "solves/s",
                "iters_per_solve": [i["iters"] for i in bi],
                "rel_residual_fp64": max(i["rel_residual"] for i in bi),
                "converged": all(i["converged"] for i in bi),
                "timed_solves": len(bt)}
        hb.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        it_o, src = golden_iters(args.workload)
        it_o = it_o or int(statistics.median(iters))
        o = oracle_rate(args.workload, wl, it_o, args.cpu_sample_iters)
        cpu = {"value": 1.0 / o["solve_s"], "unit": "solves/s", "cores": cpu_cores(),
               "kind": "oracle",
               "sample": (f"{args.cpu_sample_iters} FGMRES iterations of the FP64 numpy oracle "
                          f"on the recipe at {o['n_sample']}^{wl['dim']} ({o['wall_s']:.1f} s), "
                          f"scaled by the node ratio {o['scale']:.0f} and to a {it_o}-iteration "
                          f"solve ({'oracle count' if src else 'GPU count'})")}

    lat = sorted(times)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {mcmg.FP32: "f32", mcmg.BF16: "bf16/f32",
                  mcmg.FP32_TC: "f32 (tf32x3 tensor-core mixing)"}[prec], "data": "synthetic",
        "config": dict(config_of(args, wl, sp["restart"]), parallelism=f"replicas{world}"),
        "vcycles_per_s": sum(iters) * world / total,
        "vcycles_per_s_standalone": 1.0 / vc_s,
        "iters_per_solve": iters, "rel_residual_fp64": res, "true_rel_residual_oracle": true_res,
        "converged": conv,
        "latency_ms": {"p50": 1e3 * p50, "p99": 1e3 * p99},
        "setup_s": t_setup,
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 16 * n * 2,
                "d2h_bytes_per_step": 16 * n},
        "peaks_source": pk_src,
        "fp32_ffma_tflops_measured": ffma_peak,
        "kernel_shapes": kernel_shapes,
        "transfers": transfers,
        # one V-cycle, warm, each class timed alone: smoothing steps and
        # residuals, restrictions and prolongations, the rest (lift,
        # projection, launch gaps); and the FGMRES work per iteration beside it
        "breakdown_ms": {"vcycle": 1e3 * vc_s, "smoothing": 1e3 * t_smooth,
                         "transfers": 1e3 * t_xfer,
                         "vcycle_other": 1e3 * (vc_s - t_smooth - t_xfer),
                         "iteration": 1e3 * total / max(1, sum(iters)),
                         "krylov_and_A": 1e3 * (total / max(1, sum(iters)) - vc_s)},
    }
    if bf16:
        out["bf16"] = bf16
    if cpu:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out))
    h.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
