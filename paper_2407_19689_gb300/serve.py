"""Request loop for served OT solves on one GPU (continuous batching).

Requests arrive by a Poisson process; each one's cost matrix is built on the
device when it arrives, then it is submitted to the batch engine
(pdot_batch_submit), which admits it as memory and slots free up and advances
it together with every other resident solve.  Latency = arrival to result.
The plain baseline serves the same requests one at a time (pdot_solve in
arrival order).
"""
from __future__ import annotations

import time

import numpy as np

from . import instances as I
from . import pdot


def _materialise(r, device):
    import torch
    xs, ys, f, g = I.request_points(r)
    C = I.device_cost_from_points(torch.tensor(xs, device=device), torch.tensor(ys, device=device), r.cost,
                                  scale_to_unit=True, dtype=torch.float32)
    return C, f, g


def serve_batched(requests, device: int = 0, budget_bytes: int = 150 << 30, chunk_checks: int = 1,
                  time_scale: float = 1.0, **opts):
    """Serve `requests` (sorted by arrival) through the continuous-batching
    engine.  Returns a dict with per-request latency (s), statuses, objectives
    and the wall time."""
    b = pdot.BatchSolver(device=device, hbm_budget_bytes=budget_bytes, chunk_checks=chunk_checks, **opts)
    t0 = time.perf_counter()
    nxt = 0
    arrival = {}
    lat, status, obj, iters = {}, {}, {}, {}
    pending = len(requests)
    while pending:
        now = (time.perf_counter() - t0) / time_scale
        while nxt < len(requests) and requests[nxt].arrival_s <= now:
            r = requests[nxt]
            C, f, g = _materialise(r, f"cuda:{device}")
            tid = b.submit(C, f, g, tol=r.tol, want_plan=False)
            arrival[tid] = (nxt, t0 + r.arrival_s * time_scale)
            nxt += 1
        q, run = b.pending()
        if q == 0 and run == 0 and nxt < len(requests):
            # idle: wait for the next arrival
            wait = t0 + requests[nxt].arrival_s * time_scale - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            continue
        for tid, sol in b.poll():
            k, ta = arrival.pop(tid)
            lat[k] = time.perf_counter() - ta
            status[k] = sol.status
            obj[k] = sol.result["primal_obj"]
            iters[k] = sol.result["passes"]
            pending -= 1
    wall = time.perf_counter() - t0
    launches = b.solver.launch_count()
    b.close()
    return {"latency": lat, "status": status, "obj": obj, "iters": iters, "wall_s": wall, "launches": launches}


def serve_plain(requests, device: int = 0, time_scale: float = 1.0, **opts):
    """The same requests served one at a time in arrival order (pdot_solve)."""
    s = pdot.Solver(device=device, **opts)
    t0 = time.perf_counter()
    lat, status, obj, iters = {}, {}, {}, {}
    for k, r in enumerate(requests):
        ta = t0 + r.arrival_s * time_scale
        wait = ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        C, f, g = _materialise(r, f"cuda:{device}")
        sol = s.solve(C, f, g, tol=r.tol, want_plan=False)
        lat[k] = time.perf_counter() - ta
        status[k] = sol.status
        obj[k] = sol.result["primal_obj"]
        iters[k] = sol.result["passes"]
    wall = time.perf_counter() - t0
    s.close()
    return {"latency": lat, "status": status, "obj": obj, "iters": iters, "wall_s": wall}


def summary(res: dict, requests=None) -> dict:
    keys = sorted(res["latency"])
    lat = np.array([res["latency"][k] for k in keys])
    ok = sum(1 for v in res["status"].values() if v == pdot.OK)
    out = {"requests": int(lat.size), "ok": ok, "solves_per_s": lat.size / res["wall_s"],
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean()), "wall_s": res["wall_s"]}
    if requests is not None:
        # the three slowest requests: what sets the tail
        slow = sorted(keys, key=lambda k: -res["latency"][k])[:3]
        out["slowest"] = [{"index": k, "m": requests[k].m, "n": requests[k].n, "d": requests[k].d,
                           "cost": requests[k].cost, "tol": requests[k].tol, "latency_s": res["latency"][k],
                           "passes": res.get("iters", {}).get(k)} for k in slow]
    return out
