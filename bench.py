#!/usr/bin/env python
"""Benchmark of the GB300 PDOT path (restarted PDHG for optimal transport).

Workload (default): the 4096 x 4096 image-like instance -- a 64 x 64 pixel grid
on both sides, marginals = seeded mixtures of 3-8 Gaussian blobs (sigma 2-10 px)
plus a 1e-4 floor, cost = squared grid distance scaled to [0, 1]; FP32 cost and
plan, FP64 duals and reductions; solved from X = 0, p = q = 0 to 1e-6 relative
KKT.  One step = one full solve.  Synthetic inputs stand in for the DOTmark
images of the paper, which are not available.

Prints one JSON line (rank 0).  `value` is solves per second over all ranks
(each rank solves its own seeded instance: replicas, weak scaling).
--impl reference runs the FP64 CPU oracle instead (rank 0 only), on a bounded
sample of passes per step, scaled to the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 KKT & HBM GB/s per iter; batched solves/s, p99 latency vs plain"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "pass_kernel_traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2407_19689_gb300", "csrc", "pdot_kernels.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--grid", type=int, default=64, help="grid side G: m = n = G^2")
    ap.add_argument("--cdtype", choices=["f32", "bf16", "points"], default="f32",
                    help="storage type of the cost matrix; points: generated from the pixel coordinates in every pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="host cores the oracle baseline runs on, one independent copy each (0: all)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pass-kernel", type=int, default=0,
                    help="plan-pass kernel (pdot_options.pass_kernel; 0: the autotuner's choice) -- for profiling")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per plan tile (0: by shape) -- for profiling")
    ap.add_argument("--resident", type=int, default=0, choices=[0, 1],
                    help="grid workload: solve in the resident kernel where the plan fits (pdot_options.resident) "
                         "-- for profiling")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched-vs-plain record (256 uneven instances) out of the default line")
    ap.add_argument("--workload", choices=["grid", "batch", "serve"], default="grid",
                    help="grid: the single image-like instance (default, the headline); batch: 256 uneven "
                         "instances through the batch engine vs one instance per launch; serve: Poisson "
                         "request stream through the continuous-batching engine vs a plain FIFO server")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--certify", action="store_true",
                    help="--workload batch: certify every batched result (weak-duality bound and rounded plan)")
    ap.add_argument("--batch-detail", action="store_true",
                    help="batch workload: add each instance's size, passes and times, batched and alone")
    ap.add_argument("--requests", type=int, default=60)
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (0: the --serve-loads sweep)")
    ap.add_argument("--active-mb", type=float, default=400.0,
                    help="serving: per-pass plan megabytes the active-budget engine advances together (0: skip that server)")
    ap.add_argument("--serve-loads", default="0.5,0.8,1.1",
                    help="offered loads as fractions of the one-at-a-time server's measured capacity")
    ap.add_argument("--serve-max", type=int, default=8192, help="largest m, n of served requests")
    ap.add_argument("--step-probe", action="store_true",
                    help="per-step time decomposition: the pass alone, pass + dual update (plain launches)")
    ap.add_argument("--pass-sweep", action="store_true",
                    help="time the fused pass kernel alone over kernels x tile heights x sizes (tuning table)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def aggregate_over_ranks(elapsed_s: float, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput of replicas: every rank solved `steps` instances of
    its own; the job took the slowest rank's time (MAX over ranks)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return world * steps / elapsed_s, elapsed_s


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    try:
        with open(PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic(cost_dtype: str, grid: int, variant: int):
    """Per-launch DRAM bytes of the pass kernel from the committed ncu summary
    for this cost storage, grid and kernel variant, or None when there is no
    such record or the kernel source changed since it was captured."""
    try:
        with open(TRAFFIC) as fh:
            recs = json.load(fh)["records"]
        with open(KERNEL_SRC, "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
        for rec in recs:
            if (rec["cost_dtype"], rec["grid"], rec["kernel_variant"]) == (cost_dtype, grid, variant):
                if rec.get("kernel_source_sha256") != sha:
                    return None
                return float(rec["dram_bytes_per_launch_full_size"])
        return None
    except (OSError, KeyError, ValueError, TypeError):
        return None


def workload(grid: int, rank: int, build_cost: bool = True):
    from paper_2407_19689_gb300 import instances as I
    return I.grid_blob_instance(grid, I.seed_for(1, rank), build_cost=build_cost)


def unit_for(grid: int, tol: float) -> str:
    m = grid * grid
    return f"solves/s ({m}x{m} grid-blob OT to {tol:g} rel. KKT)"


def grid_config(args, world: int = 1) -> dict:
    """The workload description both arms print."""
    m = args.grid * args.grid
    bpe = {"f32": 20, "bf16": 18, "points": 16}[args.cdtype]
    return {"workload": f"grid{args.grid}_blobs_sqeuclid (image-like {m}x{m})", "m": m, "n": m,
            "cost_dtype": args.cdtype, "tol": args.tol, "parallelism": f"replicas x{world}",
            "l2": f"working set {m * m * bpe / 1e6:.0f} MB per pass > 126 MB L2; no flush needed"}


def oracle_period(grid: int) -> int:
    """Passes per timed oracle sample: one whole check period of a real solve
    (64 passes, then the check's two KKT evaluations) where that takes 10-30 s
    of one host core (grids up to 64 x 64); 8 passes and a check above that,
    where a pass alone takes seconds (the check's share is then larger)."""
    return 64 if grid <= 64 else 8


def oracle_sample(grid: int):
    """Seconds per PDHG pass of the FP64 oracle (single thread) on the
    workload, timed over one check period (plus the solve's initial KKT
    evaluation)."""
    import numpy as np

    import oracle
    ins = workload(grid, 0)
    C32 = ins.C.astype(np.float32).astype(np.float64)
    passes = oracle_period(grid)
    t = time.perf_counter()
    oracle.solve(C32, ins.f, ins.g, oracle.Options(tol=0.0, max_passes=passes, check_every=passes))
    return (time.perf_counter() - t) / passes


def _oracle_worker(grid: int, start, out):
    """One host core's oracle sample (run in a spawned process, which loads
    no GPU code): seconds per pass of the unchanged FP64 oracle, timed after
    every worker has built its input."""
    import oracle
    oracle.build()
    import numpy as np
    ins = workload(grid, 0)
    C32 = ins.C.astype(np.float32).astype(np.float64)
    passes = oracle_period(grid)
    start.wait()
    t = time.perf_counter()
    oracle.solve(C32, ins.f, ins.g, oracle.Options(tol=0.0, max_passes=passes, check_every=passes))
    out.put((time.perf_counter() - t) / passes)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_cores(grid: int, procs: int) -> list[float]:
    """The oracle sample on `procs` host cores at once: one independent copy
    of the same check period per process (independent solves are the unit
    of the metric), started together; seconds per pass of each copy."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    start = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(grid, start, out)) for _ in range(procs)]
    for p in ps:
        p.start()
    res = [out.get() for _ in range(procs)]
    for p in ps:
        p.join()
    return res


def cpu_record(grid: int, tol: float, p_fallback: int, unit: str, cores: int) -> dict:
    """CPU baseline: the oracle on `cores` host cores (independent copies,
    aggregate solves/s), with the one-core figure beside it."""
    sample_passes = oracle_period(grid)
    p_tol, p_src = oracle_passes_to_tol(grid, tol)
    if p_tol is None:
        p_tol, p_src = p_fallback, "pass count of this GPU solve"
    one = oracle_sample(grid)
    secs = oracle_sample_cores(grid, cores) if cores > 1 else [one]
    value = sum(1.0 / (t * p_tol) for t in secs)
    return {"value": value, "unit": unit, "cores": len(secs), "kind": "oracle",
            "one_core_value": 1.0 / (one * p_tol),
            "sample": f"{len(secs)} concurrent copies of {sample_passes} FP64 PDHG passes and one check of the "
                      f"oracle on the full instance, one per host core: {statistics.mean(secs):.3f} s/pass "
                      f"(mean over copies; {one:.3f} s/pass alone) x {p_tol} passes to tol ({p_src}); "
                      f"value = the copies' solves/s added"}


def oracle_objective(grid: int, tol: float):
    """The FP64 oracle's own objective at this tolerance on the workload
    (recorded by oracle/reference_counts.py), or None."""
    path = os.path.join(ROOT, "oracle", "reference_counts.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)[f"grid{grid}"][f"{tol:g}"]["primal_obj"])
    except (OSError, KeyError, ValueError):
        return None


def oracle_passes_to_tol(grid: int, tol: float):
    path = os.path.join(ROOT, "oracle", "reference_counts.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        return int(rec[f"grid{grid}"][f"{tol:g}"]["passes"]), "oracle's own pass count"
    except (OSError, KeyError, ValueError):
        return None, None


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    passes_per_step = oracle_period(args.grid)
    p_tol, p_src = oracle_passes_to_tol(args.grid, args.tol)
    for _ in range(args.warmup):
        oracle_sample(args.grid)
    times = [oracle_sample(args.grid) for _ in range(args.steps)]
    sec_pass = statistics.mean(times)
    if p_tol is None:
        p_tol, p_src = 5000, "assumed 5000 passes (no recorded count)"
    value = 1.0 / (sec_pass * p_tol)
    unit = unit_for(args.grid, args.tol)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_pass * passes_per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": grid_config(args, args.gpus),
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": f"{passes_per_step} FP64 PDHG passes and one restart/termination check per step "
                                   f"at full size; {sec_pass:.3f} s/pass x {p_tol} passes to tol ({p_src})"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2407_19689_gb300 import _build, pdot
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()
    pdot.load()
    dev = f"cuda:{local}"
    import ctypes

    from paper_2407_19689_gb300 import instances as I
    points = args.cdtype == "points"
    ins = workload(args.grid, rank, build_cost=not points)
    m = n = args.grid * args.grid
    unit = unit_for(args.grid, args.tol)
    if points:
        # Cost-on-the-fly: squared pixel distance / its maximum, from the
        # 2-D integer pixel coordinates (no m x n cost buffer exists).
        P = torch.tensor(I.grid_coords(args.grid), dtype=torch.float32, device=dev)
        div = float(2 * (args.grid - 1) ** 2)
        desc = pdot.PointsCostDesc(d=2, dist=pdot.DIST["sqeuclid"], xs=P.data_ptr(), ys=P.data_ptr(), divisor=div)
        cptr, ctype, ldc = ctypes.addressof(desc), pdot.POINTS, 0
    else:
        C = torch.tensor(ins.C, dtype=torch.float32, device=dev)
        ctype = pdot.F32
        if args.cdtype == "bf16":
            C = C.to(torch.bfloat16)
            ctype = pdot.BF16
        cptr, ldc = C.data_ptr(), n
    f = torch.tensor(ins.f, device=dev)
    g = torch.tensor(ins.g, device=dev)
    X = torch.empty((m, n), dtype=torch.float32, device=dev)
    p = torch.empty(m, dtype=torch.float64, device=dev)
    q = torch.empty(n, dtype=torch.float64, device=dev)
    solver = pdot.Solver(device=local, pass_kernel=args.pass_kernel, tile_rows=args.tile_rows, resident=args.resident)
    h = solver.h

    def solve_once():
        st, r = pdot.pdot_solve(h, m, n, cptr, ctype, ldc, f.data_ptr(), g.data_ptr(), args.tol,
                                X.data_ptr(), p.data_ptr(), q.data_ptr())
        if st != pdot.OK:
            raise RuntimeError(f"solve failed: {pdot.status_str(st)}")
        return r

    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else args.warmup):
        solve_once()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = pdot.pdot_launch_count(h)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    results = [solve_once() for _ in range(args.steps)]
    e1.record()
    torch.cuda.synchronize()
    launches = pdot.pdot_launch_count(h) - launches0
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    value, elapsed = aggregate_over_ranks(elapsed, args.steps, world, dist, dev)
    if dist is not None:
        dist.barrier()
    last = results[-1]
    passes = last.passes

    # Roofline of the dominant kernel: the fused plan pass, timed alone with
    # CUDA events on the library's stream, same size and launch shape.
    st, ms_pass, bytes_pass, variant = pdot.pdot_time_pass(h, m, n, cptr, ctype, ldc, f.data_ptr(),
                                                           g.data_ptr(), 50)
    peak, peak_kind = measured_peak()
    achieved = bytes_pass / (ms_pass * 1e-3) / 1e9
    traffic = recorded_traffic(args.cdtype, args.grid, variant)

    # End to end through the C ABI with host buffers (copies inside the timing).
    e2e = None
    if not args.no_e2e:
        if points:
            Ch = P.cpu().pin_memory()
            hdesc = pdot.PointsCostDesc(d=2, dist=pdot.DIST["sqeuclid"], xs=Ch.data_ptr(), ys=Ch.data_ptr(),
                                        divisor=div)
            hptr, cbytes = ctypes.addressof(hdesc), 2 * Ch.numel() * Ch.element_size()   # xs and ys
        else:
            Ch = C.cpu().pin_memory()
            hptr, cbytes = Ch.data_ptr(), Ch.numel() * Ch.element_size()
        fh = torch.tensor(ins.f).pin_memory()
        gh = torch.tensor(ins.g).pin_memory()
        Xh = torch.empty((m, n), dtype=torch.float32).pin_memory()
        ph = torch.empty(m, dtype=torch.float64).pin_memory()
        qh = torch.empty(n, dtype=torch.float64).pin_memory()
        steps_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            st, r = pdot.pdot_solve_host(h, m, n, hptr, ctype, ldc, fh.data_ptr(), gh.data_ptr(),
                                         args.tol, Xh.data_ptr(), ph.data_ptr(), qh.data_ptr())
            if st != pdot.OK:
                raise RuntimeError(f"host solve failed: {pdot.status_str(st)}")
        t_e2e = (time.perf_counter() - t0) / steps_e2e
        e2e = {"value": world / t_e2e, "unit": unit,
               "h2d_bytes_per_step": int(cbytes + fh.numel() * 8 + gh.numel() * 8),
               "d2h_bytes_per_step": int(Xh.numel() * 4 + ph.numel() * 8 + qh.numel() * 8)}

    # Certificate of the last timed result, after the timed region: the
    # optimum lies between the weak-duality bound of its row dual p and the
    # objective of the Algorithm 3 rounding of its plan (a feasible plan, up
    # to the FP32 rounding of its entries), so its objective error is bounded
    # without an exact solver.  All three numbers come from the library.
    certificate = None
    if rank == 0:
        Xr = torch.empty_like(X)
        st_r = pdot.pdot_round(h, m, n, X.data_ptr(), f.data_ptr(), g.data_ptr(), Xr.data_ptr())
        st_k, kp = pdot.pdot_kkt(h, m, n, cptr, ctype, ldc, f.data_ptr(), g.data_ptr(), Xr.data_ptr(),
                                 p.data_ptr(), q.data_ptr())
        st_b, lower = pdot.pdot_dual_bound(h, m, n, cptr, ctype, ldc, f.data_ptr(), g.data_ptr(), p.data_ptr())
        if st_r == pdot.OK and st_k == pdot.OK and st_b == pdot.OK:
            upper = kp.cx
            obj = last.primal_obj
            certificate = {"lower": lower, "upper": upper, "rel_width": (upper - lower) / abs(lower),
                           "primal_obj_rel_err_bound": max(obj - lower, upper - obj) / abs(lower),
                           "how": "lower = f.p + g.q, q_j = min_i (C_ij - p_i) (pdot_dual_bound); upper = "
                                  "<C, Algorithm 3 rounding of the returned FP32 plan> (pdot_round, pdot_kkt)"}
        del Xr

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = args.cpu_cores if args.cpu_cores > 0 else host_cores()
        cpu = cpu_record(args.grid, args.tol, passes, unit, cores)

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        # The batched workload's own record (256 uneven instances through the
        # batch engine vs one instance per launch), after the timed region.
        batch = batch_record(1e-6)

    ref_obj = oracle_objective(args.grid, args.tol) if args.cdtype == "f32" else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"{args.cdtype} cost, f32 plan, f64 duals",
            "data": "synthetic",
            "config": grid_config(args, world),
            "time_to_tol_s": elapsed / args.steps, "passes_to_tol": passes, "iters": last.iters,
            "restarts": last.restarts, "rel_kkt": last.rel_kkt, "primal_obj": last.primal_obj,
            "primal_obj_rel_err_vs_oracle": (abs(last.primal_obj - ref_obj) / abs(ref_obj)) if ref_obj else None,
            "oracle_primal_obj": ref_obj, "certificate": certificate,
            "hbm_gbs_per_iter": last.hbm_bytes / (elapsed / args.steps) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": pdot.kernel_name(variant, ctype),
                         "bytes_per_launch": bytes_pass, "ms_per_launch": ms_pass,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clk,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched and served workloads (manual runs; one JSON line each)
# ---------------------------------------------------------------------------
def batch_record(tol: float = 1e-6, count: int = 256, detail: bool = False) -> dict:
    """The batched workload: `count` instances, m and n log-uniform in
    [64, 2048] (seeded), U[0,1]^2 points, squared-Euclidean FP32 cost,
    Dirichlet(1) marginals, each solved to `tol`; once through the batch
    engine (all submitted at once) and once one instance per launch
    (pdot_solve, the same kernels).  Inputs are on the device before either
    timed region; the clocks are host wall clocks around whole runs (each
    run ends with a device synchronisation)."""
    import math

    import torch

    from paper_2407_19689_gb300 import instances as I
    from paper_2407_19689_gb300 import pdot
    dev = "cuda:0"
    sizes = I.batch_sizes(count, I.seed_for(3))
    insts = []
    for k, (m, n) in enumerate(sizes):
        ins = I.batch_instance(m, n, I.seed_for(3, k + 1))
        insts.append((torch.tensor(ins.C, dtype=torch.float32, device=dev), ins.f, ins.g))
    elems = sum(m * n for m, n in sizes)

    def batched():
        b = pdot.BatchSolver(device=0, chunk_checks=4)
        for C, f, g in insts:
            b.submit(C, f, g, tol=tol, want_plan=False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = b.run()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        launches = b.solver.launch_count()
        b.close()
        return dt, res, launches

    def plain():
        s = pdot.Solver(device=0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = [s.solve(C, f, g, tol=tol, want_plan=False) for C, f, g in insts]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        s.close()
        return dt, res

    batched()   # warm-up (graph capture, allocator pools)
    tb, rb, launches = batched()
    tp, rp = plain()
    okb = sum(1 for v in rb.values() if v.status == pdot.OK)
    okp = sum(1 for v in rp if v.status == pdot.OK)

    def sgm10(ts):
        # shifted geometric mean with shift 10 s, the paper's summary of solve times
        return math.exp(sum(math.log(t + 10.0) for t in ts) / len(ts)) - 10.0

    def geomean_gap(rs):
        # geometric mean of |<C,X> - f^T p - g^T q| over the instances, the paper's gap summary
        gs = [max(abs(r.result["gap"]), 1e-300) for r in rs]
        return math.exp(sum(math.log(x) for x in gs) / len(gs))

    objs_b = sorted((tid, v.result["primal_obj"]) for tid, v in rb.items())
    maxdiff = max(abs(a[1] - b.result["primal_obj"]) / abs(b.result["primal_obj"])
                  for a, b in zip(objs_b, rp))
    extra = {}
    if detail:
        # tickets are issued in submission order, so sorted ids follow the instances
        bres = [rb[tid] for tid in sorted(rb)]
        extra["instances"] = [{"m": m, "n": n, "batched_passes": b.result["passes"],
                               "batched_completion_s": b.result["seconds"], "plain_passes": p.result["passes"],
                               "plain_s": p.result["seconds"], "batched_obj": b.result["primal_obj"],
                               "plain_obj": p.result["primal_obj"], "batched_rel_kkt": b.result["rel_kkt"],
                               "plain_rel_kkt": p.result["rel_kkt"],
                               "batched_avg": b.result.get("returned_average"),
                               "plain_avg": p.result.get("returned_average")}
                              for (m, n), b, p in zip(sizes, bres, rp)]
    return {**extra, "workload": f"batch{count}_loguniform64-2048_dirichlet1_sqeuclid", "elements": elems, "tol": tol,
            "batched": {"seconds": tb, "solves_per_s": count / tb, "ok": okb, "gpu_launches": launches,
                        "passes": sum(v.result["passes"] for v in rb.values()),
                        "sgm10_completion_s": sgm10([v.result["seconds"] for v in rb.values()]),
                        "geomean_gap": geomean_gap(list(rb.values()))},
            "plain": {"seconds": tp, "solves_per_s": count / tp, "ok": okp,
                      "passes": sum(v.result["passes"] for v in rp),
                      "sgm10_solve_s": sgm10([v.result["seconds"] for v in rp]),
                      "geomean_gap": geomean_gap(rp),
                      "form": "pdot_solve one instance at a time, same kernels"},
            "speedup_vs_plain": tp / tb, "max_rel_obj_diff_batched_vs_plain": maxdiff}


def batch_certificates(tol: float = 1e-6, count: int = 256) -> dict:
    """The batched workload solved once through the batch engine (plans
    kept), then every result certified by the library: the optimum of its
    instance lies between the weak-duality bound of its p (pdot_dual_bound)
    and the objective of the Algorithm 3 rounding of its FP32 plan
    (pdot_round, then <C, X> by pdot_kkt).  Reports the distribution of the
    certified bounds on each result's objective error."""
    import torch

    from paper_2407_19689_gb300 import instances as I
    from paper_2407_19689_gb300 import pdot
    dev = "cuda:0"
    sizes = I.batch_sizes(count, I.seed_for(3))
    insts = []
    for k, (m, n) in enumerate(sizes):
        ins = I.batch_instance(m, n, I.seed_for(3, k + 1))
        insts.append((torch.tensor(ins.C, dtype=torch.float32, device=dev),
                      torch.tensor(ins.f, device=dev), torch.tensor(ins.g, device=dev)))
    b = pdot.BatchSolver(device=0, chunk_checks=4)
    tick = {b.submit(C, f, g, tol=tol): k for k, (C, f, g) in enumerate(insts)}
    res = b.run()
    s = pdot.Solver(device=0)
    errs, widths, ok = [], [], 0
    for tid, sol in res.items():
        C, f, g = insts[tick[tid]]
        m, n = C.shape
        if sol.status != pdot.OK:
            continue
        ok += 1
        Xr = torch.empty_like(sol.X)
        st = pdot.pdot_round(s.h, m, n, sol.X.data_ptr(), f.data_ptr(), g.data_ptr(), Xr.data_ptr())
        st2, kp = pdot.pdot_kkt(s.h, m, n, C.data_ptr(), pdot.F32, n, f.data_ptr(), g.data_ptr(), Xr.data_ptr(),
                                sol.p.data_ptr(), sol.q.data_ptr())
        st3, lower = pdot.pdot_dual_bound(s.h, m, n, C.data_ptr(), pdot.F32, n, f.data_ptr(), g.data_ptr(),
                                          sol.p.data_ptr())
        if st != pdot.OK or st2 != pdot.OK or st3 != pdot.OK:
            raise RuntimeError("certificate calls failed")
        upper, obj = kp.cx, sol.result["primal_obj"]
        widths.append((upper - lower) / abs(lower))
        errs.append(max(obj - lower, upper - obj) / abs(lower))
    s.close()
    b.close()
    errs.sort()
    widths.sort()

    def q(v, a):
        return v[min(len(v) - 1, int(a * len(v)))]

    return {"workload": f"batch{count}_loguniform64-2048_dirichlet1_sqeuclid", "tol": tol, "ok": ok,
            "certified_rel_err_bound": {"median": q(errs, 0.5), "p90": q(errs, 0.9), "max": errs[-1],
                                        "count_le_1e-6": sum(1 for e in errs if e <= 1e-6),
                                        "count_le_1e-5": sum(1 for e in errs if e <= 1e-5)},
            "interval_rel_width": {"median": q(widths, 0.5), "max": widths[-1]}}


def run_batch(args):
    from paper_2407_19689_gb300 import _build, pdot
    _build.build()
    pdot.load()
    if args.certify:
        print(json.dumps(batch_certificates(args.tol, args.batch_count)), flush=True)
        return
    rec = batch_record(args.tol, args.batch_count, args.batch_detail)
    tb = rec["batched"]["seconds"]
    line = {"metric": METRIC, "value": args.batch_count / tb, "unit": f"solves/s ({args.batch_count} uneven "
            f"instances to {args.tol:g} rel. KKT)", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": tb * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 plan/cost, f64 duals",
            "data": "synthetic",
            "config": {"workload": rec["workload"], "elements": rec["elements"], "tol": args.tol}, **rec}
    print(json.dumps(line), flush=True)


def run_serve(args):
    import numpy as np
    import torch

    from paper_2407_19689_gb300 import _build, pdot, serve
    from paper_2407_19689_gb300 import instances as I
    _build.build()
    pdot.load()
    # Capacity of the one-at-a-time server: the same requests served back to
    # back (all arrived at time 0).  Every request has a 120 s time limit.
    lim = {"time_limit_s": 120.0}
    burst = I.serve_requests(args.requests, 1e9, I.seed_for(4), hi=args.serve_max)
    capacity = len(burst) / serve.serve_plain(burst, **lim)["wall_s"]
    loads = [args.rate / capacity] if args.rate > 0.0 else [float(x) for x in args.serve_loads.split(",")]
    points = []
    for load in loads:
        rate = load * capacity
        reqs = I.serve_requests(args.requests, rate, I.seed_for(4), hi=args.serve_max)
        rb = serve.serve_batched(reqs, **lim)
        sb = serve.summary(rb, reqs)
        # the same engine with an active-bytes budget: the oldest solve keeps
        # the bandwidth, small ones fill in beside it
        sa = None
        if args.active_mb > 0:
            ra = serve.serve_batched(reqs, batch_active_bytes=int(args.active_mb * 1e6), **lim)
            sa = serve.summary(ra, reqs)
        rp = serve.serve_plain(reqs, **lim)
        sp = serve.summary(rp, reqs)
        diffs = [abs(rb["obj"][k] - rp["obj"][k]) / max(abs(rp["obj"][k]), 1e-30) for k in rb["obj"]]
        points.append({"load_vs_plain_capacity": load, "rate_per_s": rate, "continuous_batching": sb,
                       "continuous_batching_active_budget": sa, "plain_fifo": sp,
                       "p50_ratio_plain_over_batched": sp["p50_s"] / sb["p50_s"],
                       "p99_ratio_plain_over_batched": sp["p99_s"] / sb["p99_s"],
                       "p99_ratio_plain_over_active_budget": sp["p99_s"] / sa["p99_s"] if sa else None,
                       "max_rel_obj_diff_vs_plain": float(np.max(diffs)) if diffs else None})
        print(json.dumps({"progress": points[-1]}), file=sys.stderr, flush=True)
    top = points[-1]
    line = {"metric": METRIC, "value": top["continuous_batching"]["solves_per_s"], "unit": "solves/s (Poisson stream)",
            "n_gpus": 1, "steps": len(points), "warmup": 0,
            "ms_per_step": sum(p["continuous_batching"]["wall_s"] for p in points) / len(points) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 plan/cost, f64 duals",
            "data": "synthetic",
            "config": {"workload": f"serve{args.requests}_poisson_loguniform128-{args.serve_max}",
                       "plain_capacity_per_s": capacity, "admission_budget_bytes": 150 << 30,
                       "active_budget_bytes": int(args.active_mb * 1e6),
                       "value_at_load": top["load_vs_plain_capacity"]},
            "loads": points}
    print(json.dumps(line), flush=True)


def run_pass_sweep(args):
    import torch

    import ctypes

    from paper_2407_19689_gb300 import _build, pdot
    from paper_2407_19689_gb300 import instances as I
    _build.build()
    pdot.load()
    peak, _ = measured_peak()
    out = []
    for G in (64, 128):
        ins = I.grid_blob_instance(G, I.seed_for(1), build_cost=False)
        P = torch.tensor(I.grid_coords(G), device="cuda:0")
        C = torch.cdist(P, P) ** 2
        C = (C / C.max()).float()
        f = torch.tensor(ins.f, device="cuda:0")
        g = torch.tensor(ins.g, device="cuda:0")
        m = n = G * G
        for bulk in ("2", "1", "0"):
            os.environ["PDOT_PASS_BULK"] = bulk
            # tile heights: auto, fixed ones, and the one-tile-per-warp split
            # (4096^2: 54 rows; 16384^2: 864) for the grouped kernel too
            trs = (0, 32, 64, 128) if bulk == "1" else (0, 64) if bulk == "0" else \
                (0, 32, 64, 128) + ((54,) if G == 64 else (432, 864))
            for tr in trs:
                s = pdot.Solver(device=0, tile_rows=tr)
                st, ms, b, _ = pdot.pdot_time_pass(s.h, m, n, C.data_ptr(), pdot.F32, n, f.data_ptr(), g.data_ptr(),
                                                   30 if G == 64 else 10)
                s.close()
                row = {"m": m, "kernel": {"2": "bulk-group", "1": "bulk-row", "0": "register"}[bulk],
                       "tile_rows": tr or "auto",
                       "us": ms * 1e3, "GBps": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / peak}
                out.append(row)
                print(json.dumps(row), flush=True)
        # the default kernel and tiles with the compensated reduced cost
        os.environ.pop("PDOT_PASS_BULK", None)
        s = pdot.Solver(device=0, compensated_cost=1)
        st, ms, b, var = pdot.pdot_time_pass(s.h, m, n, C.data_ptr(), pdot.F32, n, f.data_ptr(), g.data_ptr(),
                                             30 if G == 64 else 10)
        s.close()
        row = {"m": m, "kernel": "compensated cost, " + {0: "register", 1: "bulk-row", 2: "bulk-group"}.get(var, "?"),
               "tile_rows": "auto", "us": ms * 1e3,
               "GBps": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / peak}
        out.append(row)
        print(json.dumps(row), flush=True)
        del C
        torch.cuda.empty_cache()
        # the same pass with the cost generated from the pixel coordinates
        # (default kernel choice: no override left over from the loop above)
        os.environ.pop("PDOT_PASS_BULK", None)
        Pf = P.float()
        cost = pdot.PointsCostDesc(d=2, dist=pdot.DIST["sqeuclid"], xs=Pf.data_ptr(), ys=Pf.data_ptr(),
                                   divisor=float(2 * (G - 1) ** 2))
        s = pdot.Solver(device=0)
        st, ms, b, var = pdot.pdot_time_pass(s.h, m, n, ctypes.addressof(cost), pdot.POINTS, 0, f.data_ptr(),
                                             g.data_ptr(), 30 if G == 64 else 10)
        s.close()
        row = {"m": m, "kernel": "generated cost, " + {0: "register", 1: "bulk-row", 2: "bulk-group"}.get(var, "?"),
               "tile_rows": "auto", "us": ms * 1e3,
               "GBps": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / peak}
        out.append(row)
        print(json.dumps(row), flush=True)
    os.environ.pop("PDOT_PASS_BULK", None)


def run_step_probe(args):
    """Device time per PDHG step at one size, split into the fused pass alone
    (pdot_time_pass) and pass + dual update with plain stream launches
    (pdot_pdhg_steps with k = 300 minus k = 0, CUDA events), for stored FP32
    and generated costs.  A diagnostic, not a bench line."""
    import ctypes
    import math

    import torch

    from paper_2407_19689_gb300 import _build, pdot
    from paper_2407_19689_gb300 import instances as I
    _build.build()
    pdot.load()
    G = args.grid
    ins = I.grid_blob_instance(G, I.seed_for(1), build_cost=False)
    P = torch.tensor(I.grid_coords(G), device="cuda:0")
    C = torch.cdist(P, P) ** 2
    C = (C / C.max()).float()
    Pf = P.float()
    desc = pdot.PointsCostDesc(d=2, dist=pdot.DIST["sqeuclid"], xs=Pf.data_ptr(), ys=Pf.data_ptr(),
                               divisor=float(2 * (G - 1) ** 2))
    m = n = G * G
    f = torch.tensor(ins.f, device="cuda:0")
    g = torch.tensor(ins.g, device="cuda:0")
    eta = 0.5 / math.sqrt(m + n)
    out = {"m": m, "n": n}
    for name, cptr, ctype, ldc in (("f32", C.data_ptr(), pdot.F32, n), ("points", ctypes.addressof(desc), pdot.POINTS, 0)):
        s = pdot.Solver(device=0)
        st, ms, _, var = pdot.pdot_time_pass(s.h, m, n, cptr, ctype, ldc, f.data_ptr(), g.data_ptr(), 50)

        def steps(k):
            X = torch.zeros((m, n), device="cuda:0")
            p = torch.zeros(m, dtype=torch.float64, device="cuda:0")
            q = torch.zeros(n, dtype=torch.float64, device="cuda:0")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            rc = pdot.pdot_pdhg_steps(s.h, m, n, cptr, ctype, ldc, f.data_ptr(), g.data_ptr(), k, eta, 1.0,
                                      X.data_ptr(), p.data_ptr(), q.data_ptr(), 0, 0, 0)
            e1.record()
            torch.cuda.synchronize()
            if rc != pdot.OK:
                raise RuntimeError(pdot.status_str(rc))
            return e0.elapsed_time(e1)

        steps(10)
        t0 = min(steps(0) for _ in range(3))
        t1 = min(steps(300) for _ in range(3))
        out[name] = {"pass_us": ms * 1e3, "kernel_variant": var, "step_us": (t1 - t0) / 300 * 1e3}
        s.close()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.step_probe:
        run_step_probe(args)
        return
    if args.pass_sweep:
        run_pass_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
