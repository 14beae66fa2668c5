#!/usr/bin/env python3
"""Benchmark of the PeTTO hot path on GB300.

One step = one PeTTO design iteration (Fig. 5 of the paper) on the chosen workload:
APT solve of the state equation to relative residual 1e-6 (warm-started from the
previous iteration's state), compliance sensitivity, design update with the volume
multiplier, Cahn-Hilliard step, modulus refresh -- every part in libpetto's kernels.

Metric: APT Gcell-sweeps/s over the whole timed design iterations (cells x sweeps /
wall time on the device), with the sweep kernel's achieved HBM bandwidth against the
measured copy peak, seconds per design iteration and sweeps per iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                  [--method apt|pt] [--max-sweeps N]

The roofline object names the sweep kernel in use (`sweep_kernel`), the bytes per node and
component of the right-hand side its refinement sweeps read (`rhs_bytes`: 2 for the FP16
copy of the two-row 3D marching kernel) and, where an ncu capture of that kernel on that
workload exists, its DRAM bytes per launch (`traffic`).  --method pt runs the same design
iterations with PT sweeps only (the plain first-order method) for comparison.

Under torchrun (N > 1) every rank runs its own replica of the workload (independent
problems: weak scaling, no data-path collective); the barrier and max-over-ranks time
use torch.distributed.  --impl reference times the FP64 CPU oracle on this host's cores
(rank 0 only), each step a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_06971_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "cantilever3d_256x128x128": lambda: W.cantilever3d(256, 128, 128),
    "cantilever2d_1024x512": lambda: W.cantilever2d(1024, 512),
    # a 2D grid larger than L2 (8.4 M nodes, 302 MB per sweep): sweeps several per pass
    "cantilever2d_4096x2048": lambda: W.cantilever2d(4096, 2048),
    "heat2d_1024x1024": lambda: W.heat2d(1024),
    "multimat3d_384x192x192_bf16": lambda: W.multimat3d(storage="bf16"),
    "multimat3d_384x192x192_fp16": lambda: W.multimat3d(storage="f16"),
    "multimat3d_384x192x192_fp32": lambda: W.multimat3d(storage="f32"),
    "cantilever3d_64x32x32": lambda: W.cantilever3d(64, 32, 32),
    "mbb_halfbeam_60x20": lambda: W.mbb_halfbeam(60, 20),
    "mbb_multimat2d_512x128": lambda: W.mbb_multimat2d(512, 128),
    "drone3d_128x64x128": lambda: W.drone3d(128, 64, 128),
    "heat2d_paper_512": lambda: W.heat2d_paper(512),
    "multimat3d_paper_256x17x85": lambda: W.multimat3d_paper(256, 17, 85),
}
BATCH_WORKLOADS = {
    "batch2d_48": lambda: W.batch2d(48),
}
DEFAULT_WORKLOAD = "cantilever3d_256x128x128"
# The paper's own loops (fixed APT/PT counts per loop) and the throughput derived from its
# RTX 3090 timings (grid points x sweeps / wall time, design steps included): vs_baseline
# for these workloads.  The MBB figure reads its "200 000 iterations" as loops.
PAPER_DERIVED_GCELL_SWEEPS = {
    "heat2d_paper_512": 25.7,
    "mbb_multimat2d_512x128": 2.98,
    "multimat3d_paper_256x17x85": 0.372,
    "drone3d_128x64x128": 1.66,
}
METRIC = "APT Gcell-sweeps/s & % HBM roofline; s/design-iter at rel.res 1e-6"

# DRAM bytes per sweep (dram__bytes_read.sum + dram__bytes_write.sum of one launch, divided
# by the sweeps it runs) of the dominant sweep kernel from one ncu capture of the workload:
# in 3D the refinement sweep of the lean two-row marching kernel, nearly all of the sweeps
# of a design iteration; in 2D a launch of four sweeps.  Keyed by workload and kernel name,
# so that any other kernel reports null; re-captured whenever that kernel changes.
NCU_TRAFFIC = {("cantilever3d_256x128x128", "tma3/zs12"): 171960576 + 64645888,
               ("cantilever2d_4096x2048", "tb2d/k4/62x48"): (169654016 + 91595520) / 4}


def sweep_bytes(spec, tsize=4, method="apt"):
    """Algorithmic bytes of one sweep: read+write of u and (APT) of w, node fields of ncomp
    components each, and one read of the modulus (cell field)."""
    fields = 4 if method == "apt" else 2
    return spec.nnodes * fields * spec.ncomp * tsize + spec.ncells * tsize


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(ms, work, device, world):
    """Whole-job aggregation across ranks: the slowest rank's time and the summed work
    (cell-sweeps).  Uses torch.distributed when world > 1 (NCCL on GPUs, gloo on CPU)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def oracle_sample(spec, n_sweeps, openmp=False):
    """Time n oracle APT sweeps (FP64; one thread, or every host core with the oracle's
    OpenMP build) on the full grid of ``spec``.  Returns seconds.  Test/benchmark
    infrastructure only: the baseline, not the path."""
    import numpy as np
    from oracle import oracle as O
    op = O.OracleProblem(spec.dim, spec.nx, spec.ny, spec.nz, h=spec.h, physics=spec.physics, nu=spec.nu,
                         loads=spec.loads, body_source=spec.body_source, boxes=spec.boxes, openmp=openmp)
    om = O.OracleMaterials(list(spec.moduli), spec.e_min, spec.penal, spec.interp)
    E = om.modulus(spec.phi0)
    F, fixed = op.load_vector(), op.fixed_mask()
    u = np.zeros(op.ndof)
    t0 = time.perf_counter()
    op.solve(E, F, fixed, u, mode=0, n_apt=n_sweeps, n_pt=0, a=spec.apt_a, b=0.25, s1=0.25, check_every=0,
             local_dt=False)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_rate(spec, budget_s, openmp):
    t1 = oracle_sample(spec, 1, openmp)
    n = max(1, min(200, int(budget_s / max(t1, 1e-6))))
    t = oracle_sample(spec, n, openmp) if n > 1 else t1
    return spec.ncells * n / t / 1e9, n, t


def cpu_baseline(spec, budget_s=12.0):
    """The FP64 oracle on the host cores: one thread, and every core (OpenMP build, when the
    host compiler has OpenMP).  ``value`` is the all-core figure."""
    from oracle import oracle as O
    grid = f"{spec.nx}x{spec.ny}x{max(spec.nz, 1)}"
    v1, n1, t1 = _oracle_rate(spec, budget_s / 2, False)
    single = {"value": v1, "unit": "Gcell-sweeps/s", "cores": 1, "kind": "oracle",
              "sample": f"{n1} FP64 oracle APT sweeps of the full {grid} grid (global pseudo-time step, "
                        f"one thread) = {t1:.1f} s"}
    cores = host_cores()
    if cores <= 1 or not O.openmp_available():
        return dict(single, single_thread=dict(single))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    vn, nn, tn = _oracle_rate(spec, budget_s / 2, True)
    return {"value": vn, "unit": "Gcell-sweeps/s", "cores": cores, "kind": "oracle",
            "sample": f"{nn} FP64 oracle APT sweeps of the full {grid} grid (global pseudo-time step, OpenMP "
                      f"on {cores} host cores) = {tn:.1f} s",
            "single_thread": single}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    from oracle import oracle as O
    spec = WORKLOADS[args.workload]()
    cores = host_cores()
    omp = cores > 1 and O.openmp_available()
    if omp:
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    n_per_step = 1
    for _ in range(args.warmup):
        oracle_sample(spec, n_per_step, omp)
    times = [oracle_sample(spec, n_per_step, omp) for _ in range(args.steps)]
    tot = sum(times)
    value = spec.ncells * n_per_step * args.steps / tot / 1e9
    par = f"cpu-openmp-{cores}threads" if omp else "cpu-1thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gcell-sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": spec.ncells, "parallelism": par,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "Gcell-sweeps/s", "cores": cores if omp else 1,
                             "kind": "oracle",
                             "sample": f"{n_per_step} FP64 oracle APT sweep of the full grid per step"
                                       + (f" (OpenMP on {cores} host cores)" if omp else " (one thread)")},
            "e2e": {"value": value, "unit": "Gcell-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_06971_gb300 import problem as PR

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS[args.workload]()
    prob = PR.Problem(spec)
    if args.kernel:
        prob.select_kernel(args.kernel)
    solve_kw = dict(tol=args.tol, max_sweeps=args.max_sweeps, check_every=spec.check_every)
    if args.method == "pt":
        solve_kw["momentum"] = 2  # the plain first-order method: PT sweeps throughout

    def design_iter():
        hist, _ = prob.optimize(1, solve_kw=solve_kw)
        return hist[-1]

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        design_iter()
    # 3D elastic FP32 grids from 2^17 nodes: the library's first solve picked the sweep kernel
    # by timing the applicable ones (petto_autotune)
    tuned = (args.warmup > 0 and spec.dim == 3 and spec.physics == W.ELASTIC and spec.precision == "f32"
             and spec.nnodes >= (1 << 17) and not args.kernel)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_idx = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gpu_idx)
    clocks.start()
    prob.profile(True)
    prob.profile_read()
    launches0 = prob.launches
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rows = [design_iter() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches = prob.launches - launches0
    kern_ms, kern_n, kern_rhs = prob.profile_read(with_rhs=True)
    prob.profile(False)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    sweeps = sum(r["sweeps"] for r in rows)
    ms_max, tot = aggregate(ms, float(sweeps) * spec.ncells, dev, world)
    value = tot / (ms_max * 1e-3) / 1e9

    peaks, peak_kind = measured_peaks()
    per_launch_ms = kern_ms / max(kern_n, 1)
    # refinement sweeps read a dense right-hand side as well (ncomp values per node; FP16 for
    # the two-row 3D marching kernel, FP32 otherwise)
    kname, rhs_b = prob.kernel_info()
    # the method's bytes per sweep (Sec. 3.2 APT/PT systems: u and w read and written, the
    # modulus read); the refinement sweeps also read a dense right-hand side, reported beside
    bytes_method = sweep_bytes(spec, method=args.method)
    bytes_rhs = (kern_rhs / max(kern_n, 1)) * spec.nnodes * spec.ncomp * rhs_b
    achieved = bytes_method / (per_launch_ms * 1e-3) / 1e9 if kern_n else None
    achieved_rhs = (bytes_method + bytes_rhs) / (per_launch_ms * 1e-3) / 1e9 if kern_n else None
    peak = float(peaks.get("hbm_gbs", 6800.0))

    # end to end through the public API: design and state in from pinned host memory,
    # one design iteration, design and state back out, every step
    P, C = spec.n_phases, spec.ncomp
    phi_h = torch.empty((P, spec.ncells), dtype=torch.float32, pin_memory=True).numpy()
    u_h = torch.empty((C, spec.nnodes), dtype=torch.float32, pin_memory=True).numpy()
    phi_h[:] = prob.get_design(dtype=np.float32)
    u_h[:] = prob.get_state(dtype=np.float32)
    torch.cuda.synchronize()
    barrier()
    e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    e_sweeps = 0
    for _ in range(e_steps):
        prob.set_design(phi_h)
        prob.set_state(u_h)
        r = design_iter()
        e_sweeps += r["sweeps"]
        phi_h[:] = prob.get_design(dtype=np.float32)
        u_h[:] = prob.get_state(dtype=np.float32)
    torch.cuda.synchronize()
    e_secs = time.perf_counter() - t0
    e_t, e_tot = aggregate(e_secs, float(e_sweeps) * spec.ncells, dev, world)
    e_value = e_tot / e_t / 1e9
    h2d = phi_h.nbytes + u_h.nbytes
    d2h = phi_h.nbytes + u_h.nbytes + 8

    line = {
        "metric": METRIC, "value": value, "unit": "Gcell-sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / PAPER_DERIVED_GCELL_SWEEPS[args.workload]
                        if args.workload in PAPER_DERIVED_GCELL_SWEEPS else None),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "cells": spec.ncells, "nodes": spec.nnodes,
                   "tol": args.tol, "method": args.method, "max_sweeps": args.max_sweeps,
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2" if sweep_bytes(spec) > 129e6 else "working set fits in L2"},
        "s_per_design_iter": ms_max * 1e-3 / args.steps,
        "sweeps_per_design_iter": sweeps / args.steps,
        "final_rel_res": rows[-1]["rel_res"], "compliance": rows[-1]["compliance"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": NCU_TRAFFIC.get((args.workload, kname)) if args.method == "apt" else None,
                     "kernel": f"{args.method} sweep", "kernel_ms": per_launch_ms,
                     "bytes_per_launch": bytes_method,
                     "rhs_bytes_per_launch": bytes_rhs, "achieved_with_rhs": achieved_rhs,
                     "frac_with_rhs": (achieved_rhs / peak) if achieved_rhs else None,
                     "rhs_sweep_fraction": kern_rhs / max(kern_n, 1), "rhs_bytes": rhs_b,
                     "sweeps_per_launch": int(kname.split("/")[1][1:]) if kname.startswith("tb2d/") else 1,
                     "sweep_kernel": kname, "sweep_kernel_choice": ("autotuned on the first solve" if tuned else
                                             ("selected" if args.kernel else "default")),
                     "peak_kind": peak_kind},
        "e2e": {"value": e_value, "unit": "Gcell-sweeps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e_steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec)
    if rank == 0:
        print(json.dumps(line))
    prob.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_time_to_design(args):
    """Time to design: the workload's whole design run (its design_steps loops from the
    initial design), wall time on the device, with the final compliance and volume."""
    import numpy as np
    import torch

    from paper_2509_06971_gb300 import problem as PR
    torch.cuda.set_device(0)
    spec = WORKLOADS[args.workload]()
    steps = args.design_steps or spec.design_steps
    prob = PR.Problem(spec)
    if args.kernel:
        prob.select_kernel(args.kernel)
    solve_kw = dict(tol=spec.tol, max_sweeps=args.max_sweeps, check_every=spec.check_every)
    warm = PR.Problem(spec)  # graph capture and first-touch outside the timed run
    warm.optimize(1, solve_kw=solve_kw)
    warm.close()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist, _ = prob.optimize(steps, solve_kw=solve_kw)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) * 1e-3
    sweeps = sum(h["sweeps"] for h in hist)
    phi = prob.get_design()
    line = {"metric": "time to design", "value": secs, "unit": "s", "higher_is_better": False,
            "workload": args.workload, "design_steps": steps, "total_sweeps": sweeps,
            "Gcell_sweeps_per_s": spec.ncells * sweeps / secs / 1e9,
            "final_compliance": hist[-1]["compliance"], "final_rel_res": hist[-1]["rel_res"],
            "final_mean_phi": [float(x) for x in phi.mean(axis=1)], "target_vol": list(spec.vol_frac),
            "max_rel_res": max(h["rel_res"] for h in hist), "data": "synthetic"}
    print(json.dumps(line))
    prob.close()
    return 0


def shard(items, rank, world):
    """The problems of a batch that rank `rank` of `world` solves: every world-th one, so
    the ranks get mixed sizes; independent problems need no collective."""
    return list(items)[rank::world]


def run_batch(args):
    """Batched workload: 48 independent 2D problems (128x64 .. 1024x512 cells) advanced
    together, one persistent launch per sweep.  A step is one design iteration of every
    problem (batched solve to 1e-6, then each problem's sensitivity, update and
    Cahn-Hilliard step).  The same design iteration run problem by problem through the
    single-problem path is timed beside it (time-to-design comparison)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_06971_gb300 import problem as PR

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_specs = BATCH_WORKLOADS[args.workload]()
    specs = shard(all_specs, rank, world)  # N > 1: the 48 problems are split across ranks
    probs = [PR.Problem(s) for s in specs]
    batch = PR.Batch(probs)
    solve_kw = dict(tol=args.tol, max_sweeps=args.max_sweeps, check_every=50)
    cells = np.array([s.ncells for s in specs], dtype=np.float64)
    nodes = np.array([s.nnodes for s in specs], dtype=np.float64)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        batch.optimize(1, solve_kw=solve_kw)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[local] if vis else str(local))
    clocks.start()
    batch.profile(True)
    batch.profile_read()
    launches0 = batch.launches
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ms_rows = []
    for _ in range(args.steps):
        m, _ = batch.optimize(1, solve_kw=solve_kw)
        ms_rows.append(m[0])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches = batch.launches - launches0
    kern_ms, kern_n = batch.profile_read()
    batch.profile(False)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    sweeps = np.array([r[:, 4] for r in ms_rows])          # [steps, n]
    work = float((sweeps * cells[None, :]).sum())
    ms_max, tot = aggregate(ms, work, dev, world)
    value = tot / (ms_max * 1e-3) / 1e9
    # algorithmic bytes of all batched sweeps in the timed region (state and modulus
    # fields of each problem for each of its sweeps; refinement right-hand sides not counted)
    per_sweep = nodes * 4 * 2 * 4 + cells * 4
    bytes_tot = float((sweeps * per_sweep[None, :]).sum())
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_tot / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None

    # time-to-design against the single-problem path: the same design iteration (same
    # designs and states) run once batched and once problem by problem
    snap = [(q.get_design(dtype=np.float32), q.get_state(dtype=np.float32)) for q in probs]
    alone_probs = [PR.Problem(s) for s in specs]
    for p, (ph, uh) in zip(alone_probs, snap):
        p.set_design(ph)
        p.set_state(uh)
        p.optimize(1, solve_kw=solve_kw)  # warm-up (graph capture)
        p.set_design(ph)
        p.set_state(uh)
    for q, (ph, uh) in zip(probs, snap):
        q.set_design(ph)
        q.set_state(uh)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    mb, _ = batch.optimize(1, solve_kw=solve_kw)
    b1.record(stream)
    torch.cuda.synchronize()
    batch_ms = b0.elapsed_time(b1)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    alone_sweeps = [p.optimize(1, solve_kw=solve_kw)[0][-1]["sweeps"] for p in alone_probs]
    a1.record(stream)
    torch.cuda.synchronize()
    alone_ms = a0.elapsed_time(a1)
    batch_sweeps = [int(x) for x in mb[0][:, 4]]
    for p in alone_probs:
        p.close()

    # end to end through the public API: designs and states in from pinned host memory,
    # one batched design iteration, designs and states back out
    hosts = []
    for q, s in zip(probs, specs):
        ph = torch.empty((s.n_phases, s.ncells), dtype=torch.float32, pin_memory=True).numpy()
        uh = torch.empty((s.ncomp, s.nnodes), dtype=torch.float32, pin_memory=True).numpy()
        ph[:] = q.get_design(dtype=np.float32)
        uh[:] = q.get_state(dtype=np.float32)
        hosts.append((ph, uh))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q, (ph, uh) in zip(probs, hosts):
        q.set_design(ph)
        q.set_state(uh)
    m, _ = batch.optimize(1, solve_kw=solve_kw)
    for q, (ph, uh) in zip(probs, hosts):
        ph[:] = q.get_design(dtype=np.float32)
        uh[:] = q.get_state(dtype=np.float32)
    torch.cuda.synchronize()
    e_secs = time.perf_counter() - t0
    e_work = float((m[0][:, 4] * cells).sum())
    e_t, e_tot = aggregate(e_secs, e_work, dev, world)
    hbytes = sum(ph.nbytes + uh.nbytes for ph, uh in hosts)

    line = {
        "metric": METRIC, "value": value, "unit": "Gcell-sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(all_specs),
                   "cells": int(sum(x.ncells for x in all_specs)), "nodes": int(sum(x.nnodes for x in all_specs)),
                   "tol": args.tol, "parallelism": f"problems sharded over {world} rank(s)",
                   "l2": "inputs larger than L2" if float(per_sweep.sum()) > 129e6 else "working set fits in L2"},
        "s_per_design_iter": ms_max * 1e-3 / args.steps,
        "sweeps_per_design_iter": {"max": float(sweeps.max()), "mean": float(sweeps.mean())},
        "single_problem_path": {"s_per_design_iter": alone_ms * 1e-3, "batched_s_per_design_iter": batch_ms * 1e-3,
                                "batched_speedup": alone_ms / batch_ms,
                                "kernel": "default single-problem 2D sweep (y-marching from 200 K nodes, node gather below)",
                                "sweeps_total": int(sum(alone_sweeps)), "batched_sweeps_total": int(sum(batch_sweeps))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel": "batched apt sweep", "kernel_ms": kern_ms / max(kern_n, 1),
                     "bytes_per_launch": bytes_tot / max(kern_n, 1), "peak_kind": peak_kind},
        "e2e": {"value": e_tot / e_t / 1e9, "unit": "Gcell-sweeps/s", "h2d_bytes_per_step": hbytes,
                "d2h_bytes_per_step": hbytes, "steps": 1},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    batch.close()
    for q in probs:
        q.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_sweeps_only(args):
    """N APT sweeps from a seeded state: few launches, for ncu captures of the sweep."""
    import torch
    from paper_2509_06971_gb300 import problem as PR
    torch.cuda.set_device(0)
    if args.workload in BATCH_WORKLOADS:
        # batched sweeps from the zero state: a tolerance no problem reaches, checks every 2
        specs = BATCH_WORKLOADS[args.workload]()
        probs = [PR.Problem(s) for s in specs]
        batch = PR.Batch(probs)
        batch.solve(tol=1e-30, max_sweeps=2, check_every=2, refine=False)
        torch.cuda.synchronize()
        batch.profile(True)
        batch.profile_read()
        batch.solve(tol=1e-30, max_sweeps=args.sweeps_only, check_every=2, refine=False)
        ms, n = batch.profile_read()
        nodes = sum(s.nnodes for s in specs)
        cells = sum(s.ncells for s in specs)
        per = ms / max(n, 1)
        print(json.dumps({"workload": args.workload, "sweeps": n, "ms_per_sweep": per,
                          "GBps": (nodes * 32 + cells * 4) / (per * 1e-3) / 1e9,
                          "Gcell_sweeps_per_s": cells / (per * 1e-3) / 1e9}))
        batch.close()
        for p in probs:
            p.close()
        return 0
    spec = WORKLOADS[args.workload]()
    prob = PR.Problem(spec)
    if args.kernel:
        prob.select_kernel(args.kernel)
    u0 = W.random_state(spec, seed=1, scale=1e-3).astype("float32")
    prob.set_state(u0)
    prob.sweep(0, 2, 0.99, 0.9, 0.75, True)
    torch.cuda.synchronize()
    prob.profile(True)
    prob.profile_read()
    prob.sweep(0, args.sweeps_only, 0.99, 0.9, 0.75, True)
    ms, n = prob.profile_read()
    per = ms / max(n, 1)
    print(json.dumps({"workload": args.workload, "sweeps": n, "ms_per_sweep": per,
                      "GBps": sweep_bytes(spec) / (per * 1e-3) / 1e9,
                      "Gcell_sweeps_per_s": spec.ncells / (per * 1e-3) / 1e9}))
    prob.close()
    return 0


def run_defects_only(args):
    """N FP64 defects F - K(E) u of the refinement (petto_residual64 on device buffers, a
    seeded FP64 state): few launches, for ncu captures of the defect kernel."""
    import ctypes
    import torch
    from paper_2509_06971_gb300 import problem as PR
    torch.cuda.set_device(0)
    spec = WORKLOADS[args.workload]()
    prob = PR.Problem(spec)
    prob.set_design(W.random_design(spec, seed=61))
    u = torch.from_numpy(W.random_state(spec, seed=62, scale=1e-2).reshape(-1)).to("cuda")
    R = torch.empty_like(u)
    r2 = ctypes.c_double(0.0)

    def defect():
        prob._ck(prob.lib.petto_residual64(prob.ctx, ctypes.c_void_p(u.data_ptr()), 1, ctypes.byref(r2),
                                           ctypes.c_void_p(R.data_ptr())))
    defect()
    t0 = time.perf_counter()
    for _ in range(args.defects_only):
        defect()
    ms = (time.perf_counter() - t0) * 1e3 / args.defects_only
    print(json.dumps({"workload": args.workload, "defects": args.defects_only, "ms_per_call": ms,
                      "note": "petto_residual64 wall time: two packing kernels and a synchronisation included",
                      "res2": r2.value}))
    prob.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-sweeps", type=int, default=20000)
    ap.add_argument("--method", choices=["apt", "pt"], default="apt",
                    help="pt: the same design iterations with PT sweeps only (the plain first-order method)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps-only", type=int, default=0,
                    help="only run this many APT sweeps of the workload (for profiler captures)")
    ap.add_argument("--defects-only", type=int, default=0,
                    help="only run this many FP64 refinement defects of the workload (for profiler captures)")
    ap.add_argument("--time-to-design", action="store_true",
                    help="time the workload's whole design run instead (one JSON line)")
    ap.add_argument("--design-steps", type=int, default=0, help="with --time-to-design: override the step count")
    ap.add_argument("--kernel", default="",
                    help="sweep kernel by name (petto_select_kernel), instead of the default or autotuned one")
    args = ap.parse_args()
    if args.sweeps_only:
        return run_sweeps_only(args)
    if args.defects_only:
        return run_defects_only(args)
    if args.time_to_design:
        return run_time_to_design(args)
    if args.impl == "reference":
        if args.workload in BATCH_WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-problem workloads"}))
            return 0
        return run_reference(args)
    if args.workload in BATCH_WORKLOADS:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
