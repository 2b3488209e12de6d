"""Throughput of the Hermite half step (DOF-updates/s) on GB300, FP64 vs mixed
precision at a stated error.

Workload: m = 3, periodic 256^3 cube, c = 1, dt = 0.4 h, a seeded N(0,1) state
(8.6 GB (FP32) / 17.2 GB (FP64) per state, far larger than the 129 MB L2, so
no L2 flush is needed between steps).  A step is one half step of the whole
grid: one kernel launch.

Every precision variant is timed on that workload, and its error at t = 1 is
measured in the same run on the precision workload (m = 2 Gaussian pulse,
sigma = 0.05, dt = 0.4 h, 128^3, 640 half steps) against the FP64 GPU path,
itself equal to the FP64 oracle to 1e-12 per half step (tests).  `value` is
the fastest variant whose measured error is at most 1e-5 (the stated bar);
every variant is listed under "variants" with its time, error and HBM
fraction, and the plain FP64 path under "fp64".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs independent replicas, one per GPU, no collectives on the
data path (the method needs none for independent simulations): "scaling":
"weak", value = all ranks' DOF-updates / max-over-ranks time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M_ORDER = 3
N_SIDE = 256
METRIC = "Hermite DOF-updates/s per half step (m=3, 256^3), FP64 vs mixed at stated error"
BAR = 1e-5          # stated relative max-norm error of a mixed variant at t = 1
CONFIG = {"workload": "m=3 periodic 256^3 cube, c=1, dt=0.4h, seeded N(0,1) state, one half step per step; "
                      "inputs 8.6 GB (FP32) / 17.2 GB (FP64) per state > L2 (no flush)",
          "global_batch": 1, "parallelism": "single", "variant": "fused",
          "error_workload": "m=2 Gaussian sigma=0.05, dt=0.4h, 128^3, t=1 (640 half steps), "
                            "relative max-norm over all components vs the FP64 GPU path"}

# Precision variants: name -> (precision, state type, arithmetic).
VARIANTS = {
    "fp32": ("fp32", "fp32", "f32"),
    "3xtf32": ("3xtf32", "fp32", "f32 + 3xTF32 tensor cores"),
    "splitbf16": ("splitbf16", "fp32", "f32 + BF16x3 tensor cores"),
    "fp32_s64": ("fp32", "fp64", "f32"),
    "hybriddf": ("hybriddf", "fp64", "double-float + f32"),
    "remainder": ("remainder", "fp64", "f32 exact-split + f32"),
    "hybrid64": ("hybrid64", "fp64", "f64 + f32"),
    "fp64": ("fp64", "fp64", "f64"),
}

# Algorithmic flop per output node of the fused half step (FMA = 2 flop, butterfly add = 1):
# x-pass 6M^4 FMA + 4M^3 adds per edge, y-pass 12M^4 + 12M^3 per face, z-pass 12M^4 + 12M^3
# per cell, both fields, M = m + 1.  Reported as a nominal ALU figure only.
FLOP_PER_NODE = {m: 2 * 30 * (m + 1) ** 4 + 28 * (m + 1) ** 3 for m in (1, 2, 3)}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu captures at 128^3 scaled by the
# node count x 8; profiles/), keyed by (variant, m, side, tile): the remainder form's tile 1
# (8 x 2 cells) and FP32's staged tile 6, the schedules the autotuner picks at 256^3.  None where
# no capture of the kernel the run timed exists.
TRAFFIC_BYTES = {("remainder", 3, 256, 1): 35.49e9, ("fp32", 3, 256, 6): 22.53e9}


def dof_per_step(m=M_ORDER, n=N_SIDE):
    return 2 * (m + 1) ** 3 * n ** 3


def bench_config(world, m=M_ORDER, side=N_SIDE):
    """The `config` object of both arms' JSON lines."""
    cfg = dict(CONFIG, global_batch=world, parallelism="replicas" if world > 1 else "single",
               dof_per_step=dof_per_step(m, side))
    if side != N_SIDE or m != M_ORDER:
        cfg["workload"] = f"m={m} periodic {side}^3 (profiling size)"
    return cfg


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the t = 1 error runs (profiling)")
    ap.add_argument("--error-side", type=int, default=128)
    ap.add_argument("--side", type=int, default=N_SIDE, help="grid side (profiling runs use a smaller one)")
    ap.add_argument("--m", type=int, default=M_ORDER)
    ap.add_argument("--tile", type=int, default=-1, help="fixed schedule of every variant (skips autotuning)")
    ap.add_argument("--zchunk", type=int, default=16)
    ap.add_argument("--variants", default=",".join(VARIANTS), help="comma list of " + ", ".join(VARIANTS))
    ap.add_argument("--legs", default="split,adjoint,taylor,advection,batch,e2e",
                    help="comma list of further legs: split (FP32 split pair), adjoint (FP32 adjoint step), "
                         "taylor (full series vs RK4 at their stability limits), advection (Table 1: 150^3, "
                         "200 time steps, m = 1..3), batch (64 seeded simulations), e2e (host buffers through "
                         "the C ABI, headline variant)")
    return ap.parse_args()


def blas_threads():
    """Threads of NumPy's BLAS as configured (threadpoolctl when present, else
    the environment, else every core)."""
    try:
        from threadpoolctl import threadpool_info
        info = [i for i in threadpool_info() if i.get("user_api") == "blas"]
        if info:
            return int(info[0]["num_threads"])
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return len(os.sched_getaffinity(0))


def oracle_rate(m, n, z_cells, max_seconds):
    """DOF-updates/s of the FP64 oracle's half step on the given output z
    layers of a seeded m, n state (repeated until max_seconds / 3)."""
    from oracle import hermite as oracle
    import hermite_inputs as HI
    h = tuple(1.0 / v for v in n)
    x = HI.random_state(m, n, seed=1)
    cells, t = 0, 0.0
    while t < max_seconds / 3 or cells == 0:
        t0 = time.perf_counter()
        oracle.half_step(x, m, h, 1.0, 0.4 * min(h), 0, z_cells=z_cells)
        t += time.perf_counter() - t0
        cells += n[0] * n[1] * len(z_cells)
        if t > max_seconds:
            break
    return cells * 2 * (m + 1) ** 3 / t, t


_ONE_CORE = """
import json, sys
sys.path.insert(0, {root!r})
import bench
v, t = bench.oracle_rate(3, (128, 128, 2), [0], {sec})
print(json.dumps({{"value": v, "seconds": t}}))
"""


def cpu_baseline(max_seconds=30.0):
    """The FP64 oracle, as it stands, on bounded samples of the workload: the
    metric's sample (one 256 x 64 band of output cells of one z-layer, m = 3,
    every host core), one core (a 128 x 128 layer, OMP/BLAS threads = 1, in a
    child process), and one z-layer of 64^3 and 128^3 grids for m = 1, 2, 3."""
    cores = len(os.sched_getaffinity(0))
    v, t = oracle_rate(M_ORDER, (N_SIDE, 64, 2), [0], max_seconds / 2)
    out = {"value": v, "unit": "DOF-updates/s", "cores": cores, "blas_threads": blas_threads(), "kind": "oracle",
           "sample": "one 256x64 band of output cells of one z-layer per call, m=3, FP64 NumPy, repeated",
           "seconds": t}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _ONE_CORE.format(root=ROOT, sec=max_seconds / 4)], env=env,
                           capture_output=True, text=True, timeout=120)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": one["value"], "cores": 1, "blas_threads": 1, "seconds": one["seconds"],
                           "sample": "one 128x128 z-layer of output cells, m=3"}
    except Exception as e:  # reported, not fatal
        out["one_core"] = {"error": str(e)[:200]}
    legs = {}
    for side in (64, 128):
        for m in (1, 2, 3):
            v, t = oracle_rate(m, (side, side, 2), [0], max_seconds / 12)
            legs[f"m={m},{side}^3"] = {"value": v, "seconds": t, "sample": f"one {side}x{side} z-layer"}
    out["legs"] = legs
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running."""

    def __init__(self):
        self.proc, self.path = None, None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(int(os.environ.get("LOCAL_RANK", 0)))],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, v, device):
    """Largest of the ranks' values (all ranks get it); v itself without a process group."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, dof_per_rank, ms_max):
    """Whole-job throughput of independent replicas: every rank advances its
    own grid of dof_per_rank values per half step; the job is as slow as its
    slowest rank."""
    return world * dof_per_rank / (ms_max * 1e-3)


def fixed_or_tuned(args, plan, x, y, zchunks=(8, 16, 32, 64), reps=2):
    """--tile fixes every leg's schedule (profiling runs); otherwise autotune."""
    from paper_1609_09841_gb300.autotune import tune
    if args.tile >= 0:
        plan.set_schedule(min(args.tile, plan.schedule_count() - 1), args.zchunk)
        return {"tile": min(args.tile, plan.schedule_count() - 1), "zchunk": args.zchunk, "ms": None}
    return tune(plan, x, y, zchunks=zchunks, reps=reps, cache=None)


def timed_steps(torch, plan, x, y, steps, warmup, clocks=None):
    """W untimed then K timed half steps (alternating parity), CUDA events on
    the launching stream; returns ms per step."""
    for k in range(warmup):
        plan.step(x, y, k % 2)
        x, y = y, x
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        plan.step(x, y, k % 2)
        x, y = y, x
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def t1_errors(torch, names, side):
    """Error at t = 1 of each variant on the precision workload (m = 2,
    Gaussian pulse sigma = 0.05 at the centre, v0 = 0, c = 1, dt = 0.4 h, side^3):
    relative max-norm over all components (and over the values of u) against
    the FP64 GPU run from the same initial state."""
    import hermite_inputs as HI
    from paper_1609_09841_gb300 import Plan
    m, n, h = 2, (side,) * 3, (1.0 / side,) * 3
    dt = 0.4 * h[0]
    nhalf = int(round(1.0 / (dt / 2)))
    x0 = torch.from_numpy(HI.gaussian_pulse(m, n, h, sigma=0.05)).cuda()

    def run(plan):
        a = x0.to(plan.torch_dtype, copy=True)
        b = torch.empty_like(a)
        for k in range(nhalf):
            plan.step(a, b, k % 2)
            a, b = b, a
        torch.cuda.synchronize()
        return a

    ref = run(Plan(m, n, h, 1.0, dt, prec="fp64", state="fp64"))
    out = {}
    for name in names:
        prec, state, _ = VARIANTS[name]
        if name == "fp64":
            out[name] = {"max_rel": 0.0, "note": "the reference run itself"}
            continue
        plan = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
        a = run(plan)
        (_, mrel, _, l2rel), rc = plan.error(a, ref, 0b111)
        (_, mrelu, _, _), _ = plan.error(a, ref, 0b001)
        out[name] = {"max_rel": mrel, "l2_rel": l2rel, "u_values_max_rel": mrelu, "finite": rc == 0}
        del a, plan
    del ref, x0
    torch.cuda.empty_cache()
    return {"grid": side, "half_steps": nhalf, "errors": out}


def run_ours(args, rank, world):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1609_09841_gb300 import Plan
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    m, n = args.m, (args.side,) * 3
    h = (1.0 / args.side,) * 3
    dt = 0.4 * h[0]
    dof = dof_per_step(m, args.side)
    legs = set(args.legs.split(",")) if args.legs else set()
    names = [v for v in args.variants.split(",") if v]
    gen = torch.Generator(device="cuda").manual_seed(1609 + rank)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):  # noqa: F811 (rank-local shorthand)
        return globals()["max_over_ranks"](dist, v, "cuda")

    # 1. errors at t = 1 (decide which variants meet the bar)
    errors = None if args.no_error else t1_errors(torch, names, args.error_side)

    # 2. time every variant on the throughput workload
    x32 = torch.randn((2, m + 1, m + 1, m + 1) + n[::-1], dtype=torch.float32, device="cuda", generator=gen)
    results, sched, clk = {}, {}, {}
    for name in names:
        prec, state, arith = VARIANTS[name]
        plan = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
        x = x32.to(plan.torch_dtype, copy=True)
        y = torch.empty_like(x)
        slow = name in ("fp64", "hybrid64")
        sched[name] = fixed_or_tuned(args, plan, x, y, zchunks=(16, 32) if slow else (16, 32, 64),
                                     reps=1 if slow else 2)
        x.copy_(x32)
        steps = max(3, args.steps // 5) if slow else args.steps
        barrier()
        clocks = ClockSampler()
        ms = timed_steps(torch, plan, x, y, steps, args.warmup if not slow else min(args.warmup, 3), clocks)
        clk[name] = clocks.stop()
        barrier()
        ms = max_over_ranks(ms)
        sbytes = 8 if state == "fp64" else 4
        bytes_alg = plan.elems * sbytes * 2          # one state read, one written
        err = errors["errors"].get(name) if errors else None
        results[name] = {"prec": prec, "state": state, "arithmetic": arith, "ms_per_step": ms, "steps": steps,
                         "value": replica_value(world, dof, ms), "hbm_gbs": bytes_alg / (ms * 1e-3) / 1e9,
                         "hbm_frac": bytes_alg / (ms * 1e-3) / 1e9 / hbm_peak, "bytes_per_step": bytes_alg,
                         "t1_max_rel": err["max_rel"] if err else None,
                         "meets_bar": (err["max_rel"] <= BAR) if err else None,
                         "schedule": {k: v for k, v in sched[name].items() if k != "ms"}}
        del plan, x, y
        torch.cuda.empty_cache()
    ms64 = results.get("fp64", {}).get("ms_per_step", float("nan"))
    for r in results.values():
        r["speedup_vs_fp64"] = ms64 / r["ms_per_step"]
    compliant = [k for k, r in results.items() if r["meets_bar"] and k != "fp64"]
    head = min(compliant, key=lambda k: results[k]["ms_per_step"]) if compliant else (
        min(results, key=lambda k: results[k]["ms_per_step"]))
    hr = results[head]
    prec, state, arith = VARIANTS[head]

    extra = {}
    plan32 = Plan(m, n, h, 1.0, dt, prec="fp32", state="fp32")
    x = x32
    y = torch.empty_like(x)
    if "fp32" in sched:
        plan32.set_schedule(sched["fp32"]["tile"], sched["fp32"]["zchunk"])
    if "e2e" in legs:
        # End to end through the C ABI with pinned host buffers, headline variant and state.
        planh = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
        if head in sched:
            planh.set_schedule(sched[head]["tile"], sched[head]["zchunk"])
        tdt = torch.float64 if state == "fp64" else torch.float32
        hx = torch.empty(planh.shape, dtype=tdt, pin_memory=True)
        hy = torch.empty(planh.shape, dtype=tdt, pin_memory=True)
        hx.copy_(x32)
        for k in range(max(1, args.warmup)):    # the host link's rate settles over the first steps
            planh.step(hx.numpy(), hy.numpy(), k % 2)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            planh.step(hx.numpy(), hy.numpy(), k % 2)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps)
        bstate = planh.elems * (8 if state == "fp64" else 4)
        extra["e2e"] = {"value": world * dof / e2e_s, "unit": "DOF-updates/s", "h2d_bytes_per_step": bstate,
                        "d2h_bytes_per_step": bstate, "seconds_per_step": e2e_s, "variant": head}
        del hx, hy, planh
    if "split" in legs:         # the two-kernel design of the paper, FP32, same workload
        plans = Plan(m, n, h, 1.0, dt, prec="fp32", state="fp32", variant="split")
        ms_split = timed_steps(torch, plans, x, y, max(3, args.steps // 4), min(args.warmup, 3))
        extra["split_fp32"] = {"value": world * dof / (max_over_ranks(ms_split) * 1e-3), "ms_per_step": ms_split,
                               "fused_fp32_speedup": ms_split / results["fp32"]["ms_per_step"]
                               if "fp32" in results else None}
        del plans
    if "adjoint" in legs:       # discrete adjoint half step, FP32, same workload
        for k in range(args.warmup + args.steps):
            if k == args.warmup:
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record()
            plan32.adjoint(x, y, k % 2)
            x, y = y, x
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record()
        torch.cuda.synchronize()
        ms_adj = e0.elapsed_time(e1) / args.steps
        extra["adjoint_fp32"] = {"value": world * dof / (max_over_ranks(ms_adj) * 1e-3), "ms_per_step": ms_adj}
    if "taylor" in legs:        # full Taylor series (q = 3(2m+1)) vs RK4, each at its own stability limit
        from paper_1609_09841_gb300 import stability_limit
        q_full = 3 * (2 * m + 1)
        legt = {}
        for lname, q in (("rk4", 4), ("full", q_full)):
            lam = stability_limit(m, q)
            dtq = 2.0 * lam * h[0]
            planq = Plan(m, n, h, 1.0, dtq, prec="fp32", state="fp32", q=q)
            if "fp32" in sched:  # the tuned schedule of the RK4 kernel (the longer series reads its zchunk)
                planq.set_schedule(sched["fp32"]["tile"] if q == 4 else 0, sched["fp32"]["zchunk"])
            msq = max_over_ranks(timed_steps(torch, planq, x, y, max(3, args.steps // 2), min(args.warmup, 3)))
            legt[lname] = {"q": q, "lam": lam, "ms_per_step": msq, "value": world * dof / (msq * 1e-3),
                           "sim_time_per_s": 0.5 * dtq / (msq * 1e-3)}
            del planq
        legt["sim_time_gain_full_vs_rk4"] = legt["full"]["sim_time_per_s"] / legt["rk4"]["sim_time_per_s"]
        extra["taylor_fp32"] = legt
    if "advection" in legs:     # the paper's own workload (Table 1): advection, 150^3, 200 time steps
        extra["advection_table1"] = run_advection(torch, rank, world, max_over_ranks, hbm_peak)
    if "batch" in legs:         # 64 seeded simulations of uneven size and order, one persistent launch per half step
        extra["batch_fp32"] = run_batch(torch, rank)
    del x32, y
    kern = {"fp32": "fused_step_kernel<float, float, ...>", "fp32_s64": "fused_step_kernel<double, float, ...>",
            "3xtf32": "tc_step_kernel<..., 3xTF32>", "splitbf16": "tc_step_kernel<..., BF16x3>",
            "hybriddf": "hybrid_step_kernel<HiDF, ...>", "hybrid64": "hybrid_step_kernel<HiF64, ...>",
            "remainder": "rem_step_kernel (m = 3: tile 0 <4, 8, 4, 512>, tile 1 <4, 8, 2, 256, 2>, tile 2 <4, 4, 4, 256, 2>)",
            "fp64": "fused_step_kernel<double, double, ...>"}
    cfg = bench_config(world, m, args.side)
    out = {
        "metric": METRIC, "value": hr["value"], "unit": "DOF-updates/s", "n_gpus": world, "steps": hr["steps"],
        "warmup": args.warmup, "ms_per_step": hr["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"hybriddf": "df32+f32", "remainder": "f32 (exact-split pairs)"}.get(head, arith.split(" ")[0]), "data": "synthetic",
        "config": cfg,
        "headline": {"variant": head, "prec": prec, "state": state, "arithmetic": arith,
                     "t1_max_rel": hr["t1_max_rel"], "bar": BAR, "meets_bar": hr["meets_bar"],
                     "speedup_vs_fp64": hr.get("speedup_vs_fp64")},
        "roofline": {"bound": "hbm", "achieved": hr["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                     "frac": hr["hbm_frac"], "traffic": TRAFFIC_BYTES.get((head, m, args.side, hr["schedule"].get("tile"))),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_launch": hr["bytes_per_step"],
                     "bytes_rule": f"one state read + one written: 2 x 2(m+1)^3 x {8 if state == 'fp64' else 4} B "
                                   f"per node x {args.side}^3 nodes",
                     "kernel": kern.get(head), "schedule": hr["schedule"],
                     "alu_nominal": {"flop_per_node": FLOP_PER_NODE[m],
                                     "tflops": FLOP_PER_NODE[m] * args.side ** 3 / (hr["ms_per_step"] * 1e-3) / 1e12,
                                     "note": "nominal: the kernel's factorised flop count, no measured peak"}},
        "variants": results,
        "errors_t1": errors,
        "fp64": results.get("fp64"),
        "e2e": extra.pop("e2e", None),
        **extra,
        "gpu_launches": hr["steps"],
        "clocks": clk.get(head),
        "clocks_by_variant": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if dist is not None:
        dist.destroy_process_group()
    return out


# Table 1 of the paper: advection on a 150^3 grid, 200 time steps (400 half
# steps), GTX 980, FP32; the number of stages is not stated there.
TABLE1_SECONDS = {1: {"monolithic": 2.09, "two_kernels": 2.42}, 2: {"monolithic": 13.77, "two_kernels": 13.77},
                  3: {"monolithic": 36.17, "two_kernels": 37.23}}


def run_advection(torch, rank, world, max_over_ranks, hbm_peak, side=150, nsteps=200):
    """Time to solution of Table 1's workload: u_t = u_x1 + u_x2 + u_x3 on a
    periodic side^3 grid, seeded N(0,1) state, FP32, the whole Taylor series
    (q = 3(2m+1)), dt = 0.9 h (a tau / h = 0.45), nsteps full steps = 2 nsteps
    half steps, fused Kronecker kernel and split pair (interpolation kernel +
    Alg. 4 loop).  Inputs 0.1-0.9 GB (> L2 from m = 2 on)."""
    from paper_1609_09841_gb300 import AdvectionPlan
    import hermite_inputs as HI
    out = {"workload": f"advection u_t = u_x1 + u_x2 + u_x3, {side}^3 periodic, {nsteps} time steps "
                       f"({2 * nsteps} half steps), FP32, q = 3(2m+1), dt = 0.9 h",
           "paper_gtx980_seconds": TABLE1_SECONDS}
    h = (1.0 / side,) * 3
    for m in (1, 2, 3):
        x0 = torch.from_numpy(HI.advection_random_state(m, (side,) * 3, seed=150 + m + 7 * rank,
                                                        dtype=np.float32)).cuda()
        row = {}
        for variant in ("fused", "split"):
            plan = AdvectionPlan(m, (side,) * 3, h, (1.0, 1.0, 1.0), 0.9 * h[0], prec="fp32", state="fp32",
                                 variant=variant)
            a, b = x0.clone(), torch.empty_like(x0)
            for k in range(4):
                plan.step(a, b, k % 2)
                a, b = b, a
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.copy_(x0)
            e0.record()
            for k in range(2 * nsteps):
                plan.step(a, b, k % 2)
                a, b = b, a
            e1.record()
            torch.cuda.synchronize()
            sec = max_over_ranks(e0.elapsed_time(e1) * 1e-3)
            half_ms = sec * 1e3 / (2 * nsteps)
            dof = (m + 1) ** 3 * side ** 3
            bytes_alg = 2 * dof * 4
            row[variant] = {"seconds_to_solution": sec, "ms_per_half_step": half_ms,
                            "value": world * dof / (half_ms * 1e-3), "unit": "DOF-updates/s",
                            "hbm_gbs_algorithmic": bytes_alg / (half_ms * 1e-3) / 1e9,
                            "hbm_frac": bytes_alg / (half_ms * 1e-3) / 1e9 / hbm_peak}
            if variant == "fused":
                # the same 2 nsteps half steps in FP64 from the same state: error of the FP32 run
                p64 = AdvectionPlan(m, (side,) * 3, h, (1.0, 1.0, 1.0), 0.9 * h[0], prec="fp64", state="fp64")
                a64, b64 = x0.double(), torch.empty(x0.shape, dtype=torch.float64, device="cuda")
                for k in range(2 * nsteps):
                    p64.step(a64, b64, k % 2)
                    a64, b64 = b64, a64
                (max_abs, max_rel, l2_abs, l2_rel), _ = plan.error(a, a64, mask=0b101)
                row["fp32_vs_fp64_end_state"] = {"max_rel_all_components": max_rel, "l2_rel": l2_rel}
                del p64, a64, b64
            del plan
        key = {"fused": "monolithic", "split": "two_kernels"}
        row["speedup_vs_paper"] = {v: TABLE1_SECONDS[m][key[v]] / row[v]["seconds_to_solution"] for v in key}
        out[f"m={m}"] = row
        del x0
    return out


def run_batch(torch, rank, nhalf=200):
    """The batched workload: 64 seeded simulations (sides from {32,48,64,96}
    per dimension, m from {1,2,3}, Gaussian pulses), FP32, 200 half steps as
    one CUDA graph of persistent launches, tile shapes and z-chunks per order
    from the autotuner."""
    import hermite_inputs as HI
    from paper_1609_09841_gb300.autotune import tune_batch
    from paper_1609_09841_gb300.batch import BatchPlan
    draw = HI.batch_draw(1609 + rank)
    sims = [{"m": d["m"], "grid": d["n"], "h": d["h"], "c": 1.0, "dt": 0.4 * min(d["h"])} for d in draw]
    bp = BatchPlan(sims, prec="fp32", state="fp32")
    a = [torch.from_numpy(HI.gaussian_pulse(d["m"], d["n"], d["h"], d["centre"], d["sigma"])).float().cuda()
         for d in draw]
    b = [torch.empty_like(t) for t in a]
    tuned = tune_batch(bp, [t.clone() for t in a], b)
    bp.run(a, b, nhalf)          # capture + first replay
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bp.run(a, b, nhalf)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dofs = sum(bp.dof(i) for i in range(len(sims)))
    return {"value": dofs * nhalf / (ms * 1e-3), "unit": "DOF-updates/s", "sims": len(sims), "half_steps": nhalf,
            "ms_total": ms, "tile": tuned["tile"], "zchunk": tuned["zchunk"], "launches": nhalf}


def run_reference(args):
    """The FP64 oracle as it stands on the host cores, W untimed then K timed
    steps, each a bounded sample of the same workload: one 256 x 64 band of
    output cells of one z-layer (m = 3)."""
    from oracle import hermite as oracle
    import hermite_inputs as HI
    n = (N_SIDE, 64, 2)
    h = (1.0 / N_SIDE,) * 3
    x = HI.random_state(M_ORDER, n, seed=1)
    for _ in range(args.warmup):
        oracle.half_step(x, M_ORDER, h, 1.0, 0.4 * h[0], 0, z_cells=[0])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.half_step(x, M_ORDER, h, 1.0, 0.4 * h[0], 0, z_cells=[0])
    t = (time.perf_counter() - t0) / args.steps
    dofs = n[0] * n[1] * 2 * (M_ORDER + 1) ** 3
    v = dofs / t
    cores = len(os.sched_getaffinity(0))
    sample = "one 256x64 band of output cells of one z-layer per step (m=3, FP64 NumPy oracle)"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.gpus),
            "cpu_baseline": {"value": v, "unit": "DOF-updates/s", "cores": cores, "blas_threads": blas_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _clean(v):
    """JSON without NaN: legs that were not run report null."""
    if isinstance(v, dict):
        return {k: _clean(x) for k, x in v.items()}
    if isinstance(v, float) and not np.isfinite(v):
        return None
    return v


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(_clean(run_reference(args))))
        return
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(_clean(out)))


if __name__ == "__main__":
    main()
