"""CPU tests of host-side logic: the replica aggregation of bench.py across
ranks (two gloo processes), and the seeded workload generators."""
import json
import math
import os
import socket

import numpy as np
import pytest

from paper_2407_19689_gb300 import instances as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]          # rank 1 is the slowest replica
    value, t = bench.aggregate_over_ranks(elapsed, steps=4, world=world, dist=dist, device="cpu")
    # each replica solves its own seeded instance
    ins = I.grid_blob_instance(8, I.seed_for(1, rank))
    q.put((rank, value, t, float(ins.f[0])))
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank_gloo():
    pytest.importorskip("torch.distributed")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, v0, t0, f0), (_, v1, t1, f1) = out
    assert t0 == t1 == 3.0                       # MAX over ranks
    assert v0 == v1 == 2 * 4 / 3.0               # all ranks' solves / slowest time
    assert f0 != f1                              # distinct seeded instances per rank


def test_aggregate_single_process():
    import bench
    v, t = bench.aggregate_over_ranks(1.5, steps=3, world=1)
    assert v == 2.0 and t == 1.5


def test_serve_requests_follow_the_recipe():
    reqs = I.serve_requests(400, rate_per_s=5.0, seed=3)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.2) < 0.05                       # Poisson rate 5/s
    assert all(128 <= r.m <= 8192 and 128 <= r.n <= 8192 for r in reqs)
    assert {r.d for r in reqs} == {2, 3, 8}
    assert {r.cost for r in reqs} == {"sqeuclid", "l1"}
    assert {r.tol for r in reqs} == {1e-4, 1e-6}
    assert all(0.5 <= r.alpha <= 2.0 for r in reqs)
    logm = np.log([r.m for r in reqs])
    assert abs(logm.mean() - 0.5 * (math.log(128) + math.log(8192))) < 0.25   # log-uniform


def test_request_points_match_request_instance():
    r = I.serve_requests(3, 1.0, seed=9, lo=16, hi=40)[1]
    xs, ys, f, g = I.request_points(r)
    ins = I.request_instance(r)
    assert np.allclose(I.cost_from_points(xs, ys, r.cost) / I.cost_from_points(xs, ys, r.cost).max(), ins.C)
    assert np.array_equal(f, ins.f) and np.array_equal(g, ins.g)
    assert abs(f.sum() - 1) < 1e-15 and abs(g.sum() - 1) < 1e-15


def test_grid_blob_instance_shapes_and_normalisation():
    ins = I.grid_blob_instance(16, I.seed_for(1))
    assert ins.C.shape == (256, 256) and abs(ins.C.max() - 1.0) < 1e-15 and ins.C.min() == 0.0
    assert abs(ins.f.sum() - 1) < 1e-14 and ins.f.min() > 0
    sizes = I.batch_sizes(256, I.seed_for(3))
    assert all(64 <= m <= 2048 and 64 <= n <= 2048 for m, n in sizes)


def _shard_main(rank, world, port, q):
    """One rank of a row-sharded PDHG step (Algorithm 2): rows [r0, r1) of C,
    X and p live on this rank; the primal step and p+ are row-local, the
    column sums of 2X+ - X are the one exchange (an all-reduce), then q+ is
    updated identically on every rank."""
    import torch
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ins = I.points_instance(37, 23, 4321)
    m, n = ins.C.shape
    rng = np.random.default_rng(9)
    X = rng.random((m, n)) / (m * n)
    p, qv = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    tau, sigma = 0.3, 0.4
    r0, r1 = m * rank // world, m * (rank + 1) // world
    # row block: the oracle's step on the block gives X+ and p+ of these rows
    Xb, pb, _ = oracle.pdhg_step(ins.C[r0:r1], ins.f[r0:r1], ins.g, X[r0:r1], p[r0:r1], qv, tau, sigma)
    part = torch.tensor((2.0 * Xb - X[r0:r1]).sum(axis=0), dtype=torch.float64)
    # fixed-order all-reduce: gather every rank's partial and add them in rank order
    parts = [torch.zeros_like(part) for _ in range(world)]
    dist.all_gather(parts, part)
    colsum = parts[0].clone()
    for t in parts[1:]:
        colsum += t
    qn = qv + sigma * (ins.g - colsum.numpy())
    q.put((rank, Xb, pb, qn))
    dist.destroy_process_group()


def test_row_sharded_step_equals_unsharded_gloo():
    """Design check of a row-sharded single instance (two gloo ranks): the
    sharded step, with one all-reduce of the column sums, reproduces the
    unsharded oracle step (X+ and p+ exactly, q+ up to the summation order)."""
    pytest.importorskip("torch.distributed")
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ins = I.points_instance(37, 23, 4321)
    m, n = ins.C.shape
    rng = np.random.default_rng(9)
    X = rng.random((m, n)) / (m * n)
    p, qv = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    Xo, po, qo = oracle.pdhg_step(ins.C, ins.f, ins.g, X, p, qv, 0.3, 0.4)
    np.testing.assert_array_equal(np.vstack([o[1] for o in out]), Xo)
    np.testing.assert_array_equal(np.concatenate([o[2] for o in out]), po)
    for o in out:
        np.testing.assert_allclose(o[3], qo, rtol=1e-13, atol=1e-15)


def _fixed_order_allreduce(vec, world, dist):
    """Sum of every rank's vector, added in rank order (the same bits on
    every rank)."""
    import torch
    part = torch.tensor(np.asarray(vec, dtype=np.float64))
    parts = [torch.zeros_like(part) for _ in range(world)]
    dist.all_gather(parts, part)
    total = parts[0].clone()
    for t in parts[1:]:
        total += t
    return total.numpy()


SHARD_PASSES = 5


def _shard_period_main(rank, world, port, q):
    """One rank of a row-sharded solve over several passes and a check.

    Rows [r0, r1) of C, X, f and p live on the rank; q and the column sums c
    of the current plan are replicated.  Per pass one all-reduce of
    [column sums of X+ - X (n) | ||X+ - X||^2 | dp . (row sums of X+ - X) |
    ||dp||^2] gives every rank the q update (2c+ - c = c + 2 dc) and the
    step-size ratio of the Sec. 5 rule; per check one all-reduce of
    [column sums of X (n) | ||r - f||^2 | dual-infeasibility^2 | <C, X> |
    f.p | ||f||^2 | ||C||_F^2] gives the KKT error of Sec. 3.1 and its
    relative measures."""
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ins = I.points_instance(37, 23, 4321)
    m, n = ins.C.shape
    rng = np.random.default_rng(9)
    X0 = rng.random((m, n)) / (m * n)
    p0, q0 = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    eta, omega = 0.05, 1.3
    tau, sigma = eta / omega, eta * omega
    r0, r1 = m * rank // world, m * (rank + 1) // world
    Cb, fb, Xb, pb, qv = ins.C[r0:r1], ins.f[r0:r1], X0[r0:r1].copy(), p0[r0:r1].copy(), q0.copy()
    g = ins.g
    c = _fixed_order_allreduce(Xb.sum(axis=0), world, dist)
    eta_bar = None
    for _ in range(SHARD_PASSES):
        Xn, pn, _ = oracle.pdhg_step(Cb, fb, g, Xb, pb, qv, tau, sigma)   # row-local X+ and p+
        dX = Xn - Xb
        dp = pn - pb
        buf = _fixed_order_allreduce(
            np.concatenate([dX.sum(axis=0), [np.sum(dX * dX), dp @ dX.sum(axis=1), dp @ dp]]), world, dist)
        dc, dx2, dpdr, dp2 = buf[:n], buf[n], buf[n + 1], buf[n + 2]
        qn = qv + sigma * (g - (c + 2.0 * dc))
        dq = qn - qv
        eta_bar = (omega * dx2 + (dp2 + dq @ dq) / omega) / (2.0 * abs(dpdr + dq @ dc))
        Xb, pb, qv, c = Xn, pn, qn, c + dc
    V = pb[:, None] + qv[None, :] - Cb
    kb = _fixed_order_allreduce(
        np.concatenate([Xb.sum(axis=0), [np.sum((Xb.sum(axis=1) - fb) ** 2), np.sum(np.where(V > 0, V * V, 0.0)),
                                        np.sum(Cb * Xb), fb @ pb, fb @ fb, np.sum(Cb * Cb)]]), world, dist)
    cx_exact = kb[:n]
    rp2 = kb[n] + np.sum((cx_exact - g) ** 2)
    rd2, cx, dual = kb[n + 1], kb[n + 2], kb[n + 3] + g @ qv
    gap = cx - dual
    rel_p = np.sqrt(rp2) / np.sqrt(kb[n + 4] + g @ g)
    rel_d = np.sqrt(rd2) / np.sqrt(kb[n + 5])
    rel_gap = abs(gap) / (abs(cx) + abs(dual))
    kkt = dict(rp2=rp2, rd2=rd2, gap=gap, kkt=np.sqrt(rp2 + rd2 + gap * gap),
               rel_kkt=max(rel_p, rel_d, rel_gap))
    q.put((rank, Xb, pb, qv, eta_bar, kkt, np.abs(c - cx_exact).max()))
    dist.destroy_process_group()


def test_row_sharded_passes_and_check_equal_unsharded_gloo():
    """Design check of a row-sharded single instance over several passes and
    a restart check (two gloo ranks, 37 rows split 18 / 19): the plan, the
    duals, the step-size ratio of the last pass and the KKT measures equal
    the unsharded oracle's up to the summation order of the exchanged sums,
    and the running column sums equal the exact column sums at the check."""
    pytest.importorskip("torch.distributed")
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_period_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ins = I.points_instance(37, 23, 4321)
    m, n = ins.C.shape
    rng = np.random.default_rng(9)
    X0 = rng.random((m, n)) / (m * n)
    p0, q0 = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    eta, omega = 0.05, 1.3
    X, p, qv, *_ = oracle.pdhg_steps(ins.C, ins.f, ins.g, X0, p0, q0, SHARD_PASSES - 1, eta, omega)
    Xn, pn, qn = oracle.pdhg_step(ins.C, ins.f, ins.g, X, p, qv, eta / omega, eta * omega)
    dX, dp, dq = Xn - X, pn - p, qn - qv
    eta_bar = (omega * np.sum(dX * dX) + (dp @ dp + dq @ dq) / omega) / (
        2.0 * abs(dp @ dX.sum(axis=1) + dq @ dX.sum(axis=0)))
    np.testing.assert_allclose(np.vstack([o[1] for o in out]), Xn, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(np.concatenate([o[2] for o in out]), pn, rtol=1e-12, atol=1e-15)
    k = oracle.kkt(ins.C, ins.f, ins.g, Xn, pn, qn)
    for o in out:
        np.testing.assert_allclose(o[3], qn, rtol=1e-12, atol=1e-15)
        assert abs(o[4] - eta_bar) <= 1e-9 * eta_bar
        assert o[6] <= 1e-15
        for key in ("rp2", "rd2", "gap", "kkt", "rel_kkt"):
            assert abs(o[5][key] - getattr(k, key)) <= 1e-10 * abs(getattr(k, key)), key
    assert out[0][4] == out[1][4] and out[0][5] == out[1][5]   # replicated decisions see the same bits


def test_recorded_traffic_is_null_once_the_kernel_source_changes(tmp_path, monkeypatch):
    """bench.py reports the ncu DRAM traffic of the pass kernel only while the
    kernel source still hashes to the value recorded with the capture."""
    import hashlib
    import json

    import bench
    src = tmp_path / "kernels.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"cost_dtype": "f32", "grid": 64, "kernel_variant": 1, "dram_bytes_per_launch_full_size": 123.0,
           "kernel_source_sha256": hashlib.sha256(src.read_bytes()).hexdigest()}
    traffic = tmp_path / "traffic.json"
    traffic.write_text(json.dumps({"records": [rec]}))
    monkeypatch.setattr(bench, "TRAFFIC", str(traffic))
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    assert bench.recorded_traffic("f32", 64, 1) == 123.0
    assert bench.recorded_traffic("bf16", 64, 1) is None      # no record for that cost storage
    assert bench.recorded_traffic("f32", 64, 2) is None       # nor for another kernel variant
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.recorded_traffic("f32", 64, 1) is None


def test_committed_traffic_record_names_its_command_and_workload():
    import json
    import bench
    recs = json.load(open(bench.TRAFFIC))["records"]
    assert recs
    for r in recs:
        assert r["command"].startswith("ncu ") and "--clock-control none" in r["command"]
        assert r["dram_bytes_per_launch_full_size"] == pytest.approx(
            r["dram_bytes_read_per_launch"] + r["dram_bytes_write_per_launch"], rel=1e-6)
        assert 0 < r["dram_bytes_per_launch_full_size"] <= 1.5 * r["algorithmic_bytes_per_launch"]


def test_measured_peak_reads_the_copy_bandwidth(tmp_path, monkeypatch):
    import json
    import bench
    peaks = tmp_path / "peaks.json"
    peaks.write_text(json.dumps({"hbm_gbs": 6790.3, "bf16_tflops": 1900.0}))
    monkeypatch.setattr(bench, "PEAKS", str(peaks))
    assert bench.measured_peak() == (6790.3, "measured")
    monkeypatch.setattr(bench, "PEAKS", str(tmp_path / "missing.json"))
    assert bench.measured_peak() == (6800.0, "fallback")


def test_oracle_sample_times_whole_check_periods():
    """The CPU baseline times the oracle over one check period (the work mix
    of a real solve): 64 passes up to 64 x 64 grids, 8 above."""
    import bench
    assert bench.oracle_period(32) == 64 and bench.oracle_period(64) == 64 and bench.oracle_period(128) == 8
    t = bench.oracle_sample(4)          # a 16 x 16 instance: 64 passes and one check
    assert 0.0 < t < 1.0


def test_cpu_baseline_runs_one_oracle_copy_per_core():
    """The CPU baseline of the default line runs the unchanged oracle as
    independent copies, one per host core, in spawned processes (no GPU code
    in them), and adds their solves/s; the one-core figure is reported
    beside it."""
    import bench
    rec = bench.cpu_record(4, 1e-4, 500, "solves/s", 2)
    assert rec["kind"] == "oracle" and rec["cores"] == 2
    assert rec["value"] > 0 and rec["one_core_value"] > 0   # (a 16 x 16 sample is too short to compare)
    assert "2 concurrent copies" in rec["sample"]
    one = bench.cpu_record(4, 1e-4, 500, "solves/s", 1)
    assert one["cores"] == 1 and one["value"] == one["one_core_value"]


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host) prints one
    JSON line with the keys the harness reads; a 16 x 16 grid keeps it short."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--grid", "4",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["value"] > 0 and rec["higher_is_better"] is True and rec["config"]["m"] == 16
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == rec["value"] and cb["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun only rank 0 runs the oracle and prints; other ranks exit 0
    without work or output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--grid", "4",
                          "--gpus", "2", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=root, env=env)
    assert out.returncode == 0 and out.stdout.strip() == "", out.stderr[-2000:]


def test_oracle_objective_record():
    """bench.py reports the headline objective's relative error against the
    FP64 oracle's own objective on the same workload, read from the committed
    record (written by oracle/reference_counts.py); None where no record exists."""
    import bench
    rec = json.load(open(os.path.join(os.path.dirname(bench.TRAFFIC), "..", "oracle", "reference_counts.json")))
    assert bench.oracle_objective(64, 1e-6) == rec["grid64"]["1e-06"]["primal_obj"]
    assert bench.oracle_objective(64, 1e-5) is None and bench.oracle_objective(7, 1e-6) is None
