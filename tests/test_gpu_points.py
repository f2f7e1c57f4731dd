"""Cost generated on the fly (c_dtype PDOT_POINTS): the plan pass, the check
and the rounding compute C_ij = dist(x_i, y_j) / divisor from coordinates
instead of reading a stored matrix (Sec. 5.1 defines the costs of the image
workloads as distances between pixel coordinates).

- k-step and KKT parity against the FP64 oracle on the oracle's own cost
  matrix built from the same (FP32) coordinates, for every distance, d = 1..8,
  ragged shapes;
- on pixel grids the generated squared distance / max is the correctly rounded
  FP32 value of the stored cost, so generated and stored solves agree bit for
  bit (plans, duals, pass counts);
- solves reach the exact LP optimum; batched generated-cost requests equal
  their single solves; host-memory coordinates; argument errors;
- full size: 16384 x 16384 grid, generated vs stored steps bit for bit, and
  the 8192 x 32768 L1 case against the oracle on sampled rows.
"""
import math

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


@pytest.fixture(scope="module")
def s32():
    s = pdot.Solver(device=0, time_limit_s=120.0)
    yield s
    s.close()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _np(t):
    return t.double().cpu().numpy()


def _points(m, n, d, seed):
    rng = np.random.default_rng(seed)
    xs = rng.random((m, d)).astype(np.float32)
    ys = rng.random((n, d)).astype(np.float32)
    f = rng.dirichlet(np.ones(m))
    g = rng.dirichlet(np.ones(n))
    return xs, ys, f / f.sum(), g / g.sum()


def _grid(G):
    return I.grid_coords(G).astype(np.float32)


CASES = [(300, 517, 3, "l1", 3.0), (129, 64, 8, "sqeuclid", 8.0), (64, 200, 2, "l2", 1.5),
         (37, 33, 5, "linf", 1.0), (1, 7, 1, "sqeuclid", 1.0), (200, 1, 4, "l1", 4.0)]


@pytest.mark.parametrize("m,n,d,dist,div", CASES)
@pytest.mark.parametrize("k", [1, 10, 100])
def test_points_pdhg_steps_match_oracle(s32, m, n, d, dist, div, k):
    xs, ys, f, g = _points(m, n, d, 7 + m + n + d)
    Co = oracle.points_cost(xs.astype(np.float64), ys.astype(np.float64), dist, div)
    rng = np.random.default_rng(k)
    X0 = (rng.random((m, n)) / (m * n)).astype(np.float32).astype(np.float64)
    p0, q0 = rng.standard_normal(m) * 0.05, rng.standard_normal(n) * 0.05
    eta = 0.5 / math.sqrt(m + n)
    gp = s32.pdhg_steps(pdot.Points(xs, ys, dist, div), f, g, X0, p0, q0, k=k, eta=eta, omega=2.3)
    o = oracle.pdhg_steps(Co, f, g, X0, p0, q0, k=k, eta=eta, omega=2.3)
    # Plans by their own norm; the duals jointly, y = [p; q]: p and q are
    # fixed only up to a shared constant (p + c, q - c), so a one-entry p can
    # be a small difference of larger numbers (m = 1 here).
    assert rel(_np(gp[0]), o[0]) < 1e-5 and rel(_np(gp[3]), o[3]) < 1e-5
    for a, b, name in [((gp[1], gp[2]), (o[1], o[2]), "y"), ((gp[4], gp[5]), (o[4], o[5]), "ybar")]:
        e = rel(np.concatenate([_np(a[0]), _np(a[1])]), np.concatenate(b))
        assert e < 1e-5, (name, e)


@pytest.mark.parametrize("m,n,d,dist,div", CASES[:4])
def test_points_kkt_matches_oracle(s32, m, n, d, dist, div):
    xs, ys, f, g = _points(m, n, d, 99 + m)
    Co = oracle.points_cost(xs.astype(np.float64), ys.astype(np.float64), dist, div)
    rng = np.random.default_rng(4)
    X = (np.outer(f, g) * rng.uniform(0.5, 1.5, (m, n))).astype(np.float32).astype(np.float64)
    p, q = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    k = s32.kkt(pdot.Points(xs, ys, dist, div), f, g, X, p, q)
    ko = oracle.kkt(Co, f, g, X, p, q)
    for key in ("rp2", "rd2", "cx", "dual", "gap", "rel_p", "rel_d", "rel_gap"):
        want = getattr(ko, key)
        assert abs(k[key] - want) <= 1e-5 * max(abs(want), 1e-12), (key, k[key], want)


@pytest.mark.parametrize("G", [16, 32])
def test_points_grid_solve_is_bit_identical_to_stored_cost(G):
    """Integer pixel coordinates: the generated squared distance divided by
    its maximum equals the stored FP32 cost entry exactly, so the two solves
    take the same steps (both in the tile kernels: generated costs do not run
    resident)."""
    ins = I.grid_blob_instance(G, I.seed_for(1, G))
    P = _grid(G)
    div = float(2 * (G - 1) ** 2)
    Cs = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    a = pdot.Solver(device=0, time_limit_s=120.0, resident=0)
    b = pdot.Solver(device=0, time_limit_s=120.0)
    ra = a.solve(Cs, ins.f, ins.g, tol=1e-6)
    rb = b.solve(pdot.Points(P, P, "sqeuclid", div), ins.f, ins.g, tol=1e-6)
    assert ra.status == pdot.OK and rb.status == pdot.OK
    assert ra.result["passes"] == rb.result["passes"]
    assert ra.result["primal_obj"] == rb.result["primal_obj"] and ra.result["rel_kkt"] == rb.result["rel_kkt"]
    assert torch.equal(ra.X, rb.X) and torch.equal(ra.p, rb.p) and torch.equal(ra.q, rb.q)
    # the byte count drops from 20 to 16 per plan entry and pass
    assert rb.result["hbm_bytes"] < 0.85 * ra.result["hbm_bytes"]
    a.close()
    b.close()


@pytest.mark.parametrize("m,n,d,dist,div", [(64, 80, 3, "l1", 3.0), (90, 70, 8, "sqeuclid", 8.0)])
def test_points_solve_reaches_exact_optimum(s32, m, n, d, dist, div):
    xs, ys, f, g = _points(m, n, d, 1234 + d)
    Co = oracle.points_cost(xs.astype(np.float64), ys.astype(np.float64), dist, div)
    opt, *_ = oracle.exact_transport(Co, f, g)
    sol = s32.solve(pdot.Points(xs, ys, dist, div), f, g, tol=1e-6)
    assert sol.status == pdot.OK, sol.result
    assert abs(sol.result["primal_obj"] - opt) / opt < 5e-6
    k = oracle.kkt(Co, f, g, _np(sol.X), _np(sol.p), _np(sol.q))
    assert k.rel_kkt <= 1.05e-6
    # reading C19: at relative KKT 1e-7 the objective is within 1e-6
    sol = s32.solve(pdot.Points(xs, ys, dist, div), f, g, tol=1e-7)
    assert sol.status == pdot.OK and abs(sol.result["primal_obj"] - opt) / opt < 1e-6, sol.result


def test_points_rounding_objective():
    xs, ys, f, g = _points(60, 45, 3, 51)
    Co = oracle.points_cost(xs.astype(np.float64), ys.astype(np.float64), "l2", 2.0)
    s = pdot.Solver(device=0, round_plan=1, time_limit_s=120.0)
    sol = s.solve(pdot.Points(xs, ys, "l2", 2.0), f, g, tol=1e-6)
    Xf = _np(sol.X)
    assert abs(sol.result["rounded_obj"] - float(np.sum(Co * Xf))) <= 1e-6 * sol.result["rounded_obj"]
    s.close()


def test_points_batch_equals_single_solves():
    cases = [(150, 97, 3, "l1", 3.0), (64, 256, 2, "sqeuclid", 2.0), (200, 130, 8, "sqeuclid", 8.0)]
    bs = pdot.BatchSolver(device=0, time_limit_s=120.0)
    costs, tickets = {}, {}
    for i, (m, n, d, dist, div) in enumerate(cases):
        xs, ys, f, g = _points(m, n, d, 300 + i)
        cost = pdot.Points(xs, ys, dist, div)
        costs[i] = (cost, f, g)
        tickets[bs.submit(cost, f, g, tol=1e-6)] = i
        # a stored-cost request in the same batch
        ins = I.batch_instance(m, n, 400 + i)
        tickets[bs.submit(torch.tensor(ins.C, dtype=torch.float32, device=DEV), ins.f, ins.g, tol=1e-6)] = -1
    res = bs.run()
    for tid, i in tickets.items():
        assert res[tid].status == pdot.OK
        if i < 0:
            continue
        # the single solve with the tile height and pass kernel the batch ran
        single = pdot.Solver(device=0, tile_rows=res[tid].result["tile_rows"], pass_kernel=2, time_limit_s=120.0)
        cost, f, g = costs[i]
        a, b = res[tid], single.solve(cost, f, g, tol=1e-6)
        single.close()
        assert a.result["passes"] == b.result["passes"] and a.result["primal_obj"] == b.result["primal_obj"]
        assert torch.equal(a.X, b.X) and torch.equal(a.p, b.p)
    bs.close()
    single.close()


def test_points_host_solve_equals_device_solve(s32):
    xs, ys, f, g = _points(70, 90, 3, 77)
    dev = s32.solve(pdot.Points(xs, ys, "l1", 3.0), f, g, tol=1e-5)
    desc = pdot.PointsCostDesc(d=3, dist=pdot.DIST["l1"], xs=xs.ctypes.data, ys=ys.ctypes.data, divisor=3.0)
    import ctypes
    X = np.empty((70, 90), dtype=np.float32)
    p, q = np.empty(70), np.empty(90)
    st, r = pdot.pdot_solve_host(s32.h, 70, 90, ctypes.addressof(desc), pdot.POINTS, 0, f.ctypes.data,
                                 g.ctypes.data, 1e-5, X.ctypes.data, p.ctypes.data, q.ctypes.data)
    assert st == pdot.OK
    assert r.passes == dev.result["passes"] and r.primal_obj == dev.result["primal_obj"]
    assert np.array_equal(X, dev.X.cpu().numpy())


def test_points_argument_errors(s32):
    xs, ys, f, g = _points(8, 9, 2, 5)
    for kw in [dict(divisor=0.0), dict(divisor=float("inf"))]:
        with pytest.raises(pdot.PdotError) as e:
            s32.solve(pdot.Points(xs, ys, "l1", **kw), f, g, tol=1e-4)
        assert e.value.status == pdot.ERR_ARG
    with pytest.raises(pdot.PdotError) as e:
        s32.solve(pdot.Points(np.zeros((8, 9), np.float32), np.zeros((9, 9), np.float32)), f, g, tol=1e-4)
    assert e.value.status == pdot.ERR_ARG   # d = 9 > 8
    s64 = pdot.Solver(device=0, x_dtype=pdot.F64)
    with pytest.raises(pdot.PdotError) as e:
        s64.solve(pdot.Points(xs, ys), f, g, tol=1e-4)
    assert e.value.status == pdot.ERR_ARG   # generated costs need FP32 plans
    s64.close()


def test_points_fullsize_grid128_steps_bit_identical_to_stored():
    """16384 x 16384: four PDHG steps with the generated cost equal the steps
    with the stored FP32 cost bit for bit (same kernel family, same tiles)."""
    G = 128
    ins = I.grid_blob_instance(G, I.seed_for(2), build_cost=False)
    P = torch.tensor(_grid(G), device=DEV)
    Cs = torch.cdist(P.double(), P.double()) ** 2
    Cs = (Cs / Cs.max()).float()
    m = n = G * G
    eta = 0.7 / math.sqrt(m + n)
    z = (torch.zeros((m, n), device=DEV), torch.zeros(m, dtype=torch.float64, device=DEV),
         torch.zeros(n, dtype=torch.float64, device=DEV))
    s = pdot.Solver(device=0)
    A = s.pdhg_steps(Cs, ins.f, ins.g, *z, k=4, eta=eta)
    del Cs
    torch.cuda.empty_cache()
    B = s.pdhg_steps(pdot.Points(P, P, "sqeuclid", float(2 * (G - 1) ** 2)), ins.f, ins.g, *z, k=4, eta=eta)
    for a, b in zip(A, B):
        assert torch.equal(a, b)
    s.close()


def test_points_fullsize_rect_l1_sampled_rows():
    """8192 x 32768, L1 distance between uniform points in [0,1]^3 divided by
    3, generated on the fly: one step from a GPU iterate, checked on sampled
    rows against the oracle (primal update and p+ are row-local), and q+
    against the dual update with the full column sums."""
    m, n = 8192, 32768
    rng = np.random.default_rng(I.seed_for(2, 1))
    xs, ys = rng.random((m, 3)).astype(np.float32), rng.random((n, 3)).astype(np.float32)
    f = rng.dirichlet(np.ones(m))
    g = rng.dirichlet(np.ones(n))
    f, g = f / f.sum(), g / g.sum()
    cost = pdot.Points(xs, ys, "l1", 3.0)
    s = pdot.Solver(device=0)
    eta = 0.7 / math.sqrt(m + n)
    z = (torch.zeros((m, n), device=DEV), torch.zeros(m, dtype=torch.float64, device=DEV),
         torch.zeros(n, dtype=torch.float64, device=DEV))
    X2, p2, q2, *_ = s.pdhg_steps(cost, f, g, *z, k=3, eta=eta)
    X3, p3, q3, *_ = s.pdhg_steps(cost, f, g, X2, p2, q2, k=1, eta=eta)
    S = np.sort(np.random.default_rng(5).choice(m, 48, replace=False))
    St = torch.tensor(S, device=DEV)
    Cs = oracle.points_cost(xs[S].astype(np.float64), ys.astype(np.float64), "l1", 3.0)
    X2s = X2.index_select(0, St).double().cpu().numpy()
    Xo, po, _ = oracle.pdhg_step(Cs, f[S], np.full(n, 1.0 / n) * f[S].sum(), X2s,
                                 p2.index_select(0, St).cpu().numpy(), q2.cpu().numpy(), eta, eta)
    X3s = X3.index_select(0, St).double().cpu().numpy()
    assert np.linalg.norm(X3s - Xo) <= 1e-5 * np.linalg.norm(Xo) + 1e-12
    np.testing.assert_allclose(p3.index_select(0, St).cpu().numpy(), po, rtol=1e-5, atol=1e-12)
    c2, c3 = X2.double().sum(0), X3.double().sum(0)
    q_expect = q2 + eta * (torch.tensor(g, device=DEV) - (2.0 * c3 - c2))
    assert (torch.linalg.norm(q3 - q_expect) / torch.linalg.norm(q_expect)).item() < 1e-5
    s.close()


def test_points_grouped_kernel(monkeypatch):
    """The grouped bulk kernel (4-row stages; the autotuner's pick for large
    shapes) with generated costs: bit-identical to it with the stored cost on
    a pixel grid, and k-step parity with the oracle on random points."""
    monkeypatch.setenv("PDOT_PASS_BULK", "2")
    G = 32
    ins = I.grid_blob_instance(G, I.seed_for(1, 7))
    P = _grid(G)
    div = float(2 * (G - 1) ** 2)
    a = pdot.Solver(device=0, time_limit_s=120.0)
    b = pdot.Solver(device=0, time_limit_s=120.0)
    ra = a.solve(torch.tensor(ins.C, dtype=torch.float32, device=DEV), ins.f, ins.g, tol=1e-6)
    rb = b.solve(pdot.Points(P, P, "sqeuclid", div), ins.f, ins.g, tol=1e-6)
    assert ra.status == pdot.OK and rb.status == pdot.OK
    assert ra.result["passes"] == rb.result["passes"] and torch.equal(ra.X, rb.X) and torch.equal(ra.p, rb.p)
    Pd = torch.tensor(P, device=DEV)
    desc = pdot.PointsCostDesc(d=2, dist=0, xs=Pd.data_ptr(), ys=Pd.data_ptr(), divisor=div)
    import ctypes
    f = torch.tensor(ins.f, device=DEV)
    g = torch.tensor(ins.g, device=DEV)
    st, _, _, variant = pdot.pdot_time_pass(b.h, G * G, G * G, ctypes.addressof(desc), pdot.POINTS, 0,
                                            f.data_ptr(), g.data_ptr(), 3)
    assert st == pdot.OK and variant == 2
    a.close()
    b.close()
    s = pdot.Solver(device=0)
    m, n = 300, 517
    xs, ys, f, g = _points(m, n, 3, 4242)
    Co = oracle.points_cost(xs.astype(np.float64), ys.astype(np.float64), "l1", 3.0)
    rng = np.random.default_rng(3)
    X0 = (rng.random((m, n)) / (m * n)).astype(np.float32).astype(np.float64)
    p0, q0 = rng.standard_normal(m) * 0.05, rng.standard_normal(n) * 0.05
    eta = 0.5 / math.sqrt(m + n)
    gp = s.pdhg_steps(pdot.Points(xs, ys, "l1", 3.0), f, g, X0, p0, q0, k=20, eta=eta, omega=1.7)
    o = oracle.pdhg_steps(Co, f, g, X0, p0, q0, k=20, eta=eta, omega=1.7)
    assert rel(_np(gp[0]), o[0]) < 1e-5 and rel(_np(gp[3]), o[3]) < 1e-5
    assert rel(np.concatenate([_np(gp[1]), _np(gp[2])]), np.concatenate([o[1], o[2]])) < 1e-5
    s.close()
