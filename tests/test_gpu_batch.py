"""GPU tests of the batch engine (continuous batching): every instance's
result in a batch equals its single-instance solve (the same kernels, the
same per-instance tiles and fixed-order reductions), alone or in any mix,
whenever it joins; cancellation, admission by budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2407_19689_gb300 import instances as I  # noqa: E402
from paper_2407_19689_gb300 import pdot  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    pdot.load(build_if_missing=True)


def _inst(k):
    sizes = [(64, 64), (130, 97), (257, 300), (1, 9), (40, 333), (512, 128), (77, 77), (300, 41)]
    m, n = sizes[k % len(sizes)]
    ins = I.points_instance(m, n, 7000 + k, marginals="dirichlet", alpha=1.0)
    return torch.tensor(ins.C, dtype=torch.float32, device=DEV), ins.f, ins.g


def _same(a, b):
    ra, rb = a.result, b.result
    assert ra["status"] == rb["status"] == pdot.OK
    assert ra["passes"] == rb["passes"] and ra["restarts"] == rb["restarts"]
    assert ra["primal_obj"] == rb["primal_obj"] and ra["rel_kkt"] == rb["rel_kkt"]
    assert torch.equal(a.X, b.X) and torch.equal(a.p, b.p) and torch.equal(a.q, b.q)


@pytest.mark.parametrize("resident", [1, 0])
def test_batch_equals_single_solves(resident):
    # Resident instances (a thread-block cluster each) compute in an order
    # fixed by their shape; the others run in tiles the batch engine sizes
    # from their shape (16 to 64 rows) with the per-row bulk pass kernel.  A
    # single solve in the same kernel with the same tiles reduces in the same
    # order and must match bit for bit.
    batch = pdot.BatchSolver(device=0, time_limit_s=120.0, resident=resident)
    insts = [_inst(k) for k in range(12)]
    ids = [batch.submit(C, f, g, tol=1e-6) for C, f, g in insts]
    res = batch.run()
    assert sorted(res) == sorted(ids)
    for tid, (C, f, g) in zip(ids, insts):
        tr = res[tid].result["tile_rows"]
        if resident:
            assert tr == 0   # every instance here fits a cluster
            single = pdot.Solver(device=0, time_limit_s=120.0, resident=1)
        else:
            assert 16 <= tr <= 64 and tr % 2 == 0
            single = pdot.Solver(device=0, time_limit_s=120.0, tile_rows=tr, pass_kernel=2, resident=0)
        _same(res[tid], single.solve(C, f, g, tol=1e-6))
        single.close()
        opt, *_ = oracle.exact_transport(C.double().cpu().numpy(), f, g)
        assert abs(res[tid].result["primal_obj"] - opt) / opt < 5e-6
    batch.close()


def test_batched_fp32_objective_within_1e6_of_exact_optimum():
    """FP32-plan solves in the batch engine, stopped at relative KKT 1e-7
    (reading C19), land within 1e-6 of the exact LP optimum of Eq. (1) --
    the FP64 oracle's accuracy at the same tolerance -- and the FP64 oracle
    measures the returned point at the tolerance."""
    batch = pdot.BatchSolver(device=0, time_limit_s=120.0)
    insts = [_inst(k) for k in range(8)]
    ids = [batch.submit(C, f, g, tol=1e-7) for C, f, g in insts]
    res = batch.run()
    for tid, (C, f, g) in zip(ids, insts):
        r = res[tid]
        assert r.status == pdot.OK, r.result
        Co = C.double().cpu().numpy()
        opt, *_ = oracle.exact_transport(Co, f, g)
        assert abs(r.result["primal_obj"] - opt) / opt < 1e-6, (Co.shape, r.result)
        k = oracle.kkt(Co, f, g, r.X.double().cpu().numpy(), r.p.cpu().numpy(), r.q.cpu().numpy())
        assert k.rel_kkt <= 1.05e-7
    batch.close()


def test_continuous_admission_alone_vs_mix():
    """Requests submitted while others run join at a chunk boundary; each
    result equals the same request solved alone."""
    batch = pdot.BatchSolver(device=0, time_limit_s=120.0, chunk_checks=1)
    alone = pdot.BatchSolver(device=0, time_limit_s=120.0, chunk_checks=1)
    insts = [_inst(k) for k in range(8)]
    ids = [batch.submit(*insts[k], tol=1e-6) for k in range(3)]
    got = {}
    for tid, sol in batch.poll():
        got[tid] = sol
    ids += [batch.submit(*insts[k], tol=1e-6) for k in range(3, 6)]
    for tid, sol in batch.poll():
        got[tid] = sol
    ids += [batch.submit(*insts[k], tol=1e-4 if k == 6 else 1e-6) for k in range(6, 8)]
    got.update(batch.run())
    for k, tid in enumerate(ids):
        a = alone.submit(*insts[k], tol=1e-4 if k == 6 else 1e-6)
        ra = alone.run()
        _same(got[tid], ra[a])
    batch.close()
    alone.close()


def test_cancel_and_budget():
    b = pdot.BatchSolver(device=0, hbm_budget_bytes=64 << 20, time_limit_s=60.0)
    C, f, g = _inst(2)
    t1 = b.submit(C, f, g, tol=1e-9)
    t2 = b.submit(C, f, g, tol=1e-6)
    assert b.cancel(t1) == pdot.OK
    res = b.run()
    assert res[t1].status == pdot.CANCELLED and res[t2].status == pdot.OK
    big = torch.zeros((4096, 4096), dtype=torch.float32, device=DEV)
    fb = np.full(4096, 1 / 4096)
    with pytest.raises(pdot.PdotError) as e:
        b.submit(big, fb, fb)
    assert e.value.status == pdot.BUSY
    b.close()


def test_batch_rejects_bad_marginals_on_device():
    b = pdot.BatchSolver(device=0, time_limit_s=60.0)
    C, f, g = _inst(1)
    t_bad = b.submit(C, f, g * 2.0)
    t_ok = b.submit(C, f, g, tol=1e-4)
    res = b.run()
    assert res[t_bad].status == pdot.ERR_ARG and res[t_ok].status == pdot.OK
    b.close()


@pytest.mark.parametrize("active_bytes", [1, 3 << 20])
def test_active_bytes_policy_keeps_results(active_bytes):
    """With an active-bytes budget a chunk advances the oldest instance and the
    younger ones that fit; paused instances resume later.  Each result still
    equals the same request in an unrestricted batch (1 byte: one instance at
    a time, in admission order)."""
    free = pdot.BatchSolver(device=0, time_limit_s=120.0, chunk_checks=1)
    pol = pdot.BatchSolver(device=0, time_limit_s=120.0, chunk_checks=1, batch_active_bytes=active_bytes)
    insts = [_inst(k) for k in range(6)]
    a = [free.submit(C, f, g, tol=1e-6) for C, f, g in insts]
    b = [pol.submit(C, f, g, tol=1e-6) for C, f, g in insts]
    ra, rb = free.run(), pol.run()
    for ta, tb in zip(a, b):
        _same(ra[ta], rb[tb])
    free.close()
    pol.close()


def test_batch_time_limit_returns_the_current_iterate():
    """A batch instance past its time limit is stopped at its next restart
    check and returns the current iterate with that iterate's own KKT
    measures (PDOT_TIMEOUT), as pdot_solve does."""
    ins = I.points_instance(300, 517, 81)
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    b = pdot.BatchSolver(device=0, time_limit_s=1e-9)
    t = b.submit(C, ins.f, ins.g, tol=1e-9)
    sol = b.run()[t]
    b.close()
    r = sol.result
    assert sol.status == pdot.TIMEOUT and r["returned_average"] == 0
    assert r["passes"] > 0 and r["passes"] % 64 == 0
    X, p, q = (t_.double().cpu().numpy() for t_ in (sol.X, sol.p, sol.q))
    k = oracle.kkt(ins.C.astype(np.float32).astype(np.float64), ins.f, ins.g, X, p, q)
    assert abs(k.rel_kkt - r["rel_kkt"]) <= 1e-4 * k.rel_kkt
    assert abs(k.cx - r["primal_obj"]) <= 1e-6 * abs(k.cx)
