"""The resident kernel (pdot_options.resident = 1: one thread-block cluster
per instance, the plan and the average's deviation in shared memory, whole
check periods of Algorithm 2 per launch), on the GPU:

- k steps of Algorithm 2 against the FP64 oracle, element by element, on
  shapes with fewer rows than CTAs, one column, ragged column strips and the
  largest plan that fits;
- full solves against the exact optimum, the reported KKT against the
  oracle's KKT of the returned point, the same results as the tile kernels'
  to the tolerance;
- the fit rule (an instance just too large runs in tiles);
- the batch engine with resident and tile instances mixed: each result the
  same alone and in the mix, bit for bit.
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


def _np(t):
    return t.double().cpu().numpy()


def _rand_state(m, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 2.0 / (m * n), (m, n)) * (rng.random((m, n)) < 0.6)
    return X, rng.normal(0.0, 0.05, m), rng.normal(0.0, 0.05, n)


# (m, n): fewer rows than the cluster's CTAs; a single column; ragged strips
# (n not a multiple of 128) with more strips than one warp per strip; the
# largest square plan that fits a cluster.
SHAPES = [(5, 300), (700, 1), (130, 517), (60, 2100), (430, 430)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("k", [1, 37])
def test_resident_steps_match_oracle(m, n, k):
    ins = I.points_instance(m, n, 3100 + m + n)
    res = pdot.Solver(device=0, resident=1)
    assert pdot.pdot_resident_fits(m, n) == 1
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    Co = _np(C)
    eta = 0.5 / math.sqrt(m + n)
    for start, omega in [("zero", 1.0), ("rand", 2.3)]:
        X0, p0, q0 = (np.zeros((m, n)), np.zeros(m), np.zeros(n)) if start == "zero" else _rand_state(m, n, k)
        X0 = X0.astype(np.float32).astype(np.float64)
        g = res.pdhg_steps(C, ins.f, ins.g, X0, p0, q0, k=k, eta=eta, omega=omega)
        o = oracle.pdhg_steps(Co, ins.f, ins.g, X0, p0, q0, k=k, eta=eta, omega=omega)
        for a, b, name in zip(g, o, ("X", "p", "q", "Xbar", "pbar", "qbar")):
            a = _np(a)
            scale = max(float(np.max(np.abs(b))), 1e-300)
            assert float(np.max(np.abs(a - b))) <= 1e-5 * scale, (name, start)
    res.close()


def test_resident_steps_bf16_cost():
    m, n = 200, 333
    ins = I.points_instance(m, n, 3300)
    s = pdot.Solver(device=0, resident=1)
    C = torch.tensor(ins.C, dtype=torch.bfloat16, device=DEV)
    z = (np.zeros((m, n)), np.zeros(m), np.zeros(n))
    eta = 0.5 / math.sqrt(m + n)
    g = s.pdhg_steps(C, ins.f, ins.g, *z, k=40, eta=eta)
    o = oracle.pdhg_steps(_np(C), ins.f, ins.g, *z, k=40, eta=eta)
    for a, b in zip(g, o):
        a = _np(a)
        assert float(np.max(np.abs(a - b))) <= 1e-5 * max(float(np.max(np.abs(b))), 1e-300)
    s.close()


@pytest.mark.parametrize("m,n,seed", [(64, 64, I.seed_for(0)), (90, 47, 11), (33, 150, 12), (7, 260, 13)])
def test_resident_solve_reaches_exact_optimum(m, n, seed):
    ins = I.points_instance(m, n, seed, marginals="dirichlet")
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    Co = _np(C)
    opt, *_ = oracle.exact_transport(Co, ins.f, ins.g)
    r1 = pdot.Solver(device=0, time_limit_s=120.0, resident=1)
    r0 = pdot.Solver(device=0, time_limit_s=120.0)
    for tol, bound in [(1e-6, 5e-6), (1e-7, 1e-6)]:
        a = r1.solve(C, ins.f, ins.g, tol=tol)
        b = r0.solve(C, ins.f, ins.g, tol=tol)
        assert a.status == pdot.OK and b.status == pdot.OK
        assert a.result["tile_rows"] == 0 and b.result["tile_rows"] > 0   # resident / tiles
        assert abs(a.result["primal_obj"] - opt) / opt < bound, (tol, a.result)
        # the FP64 oracle's KKT of the returned point: within the tolerance,
        # and the device's report agrees to a tenth of it (the device sums the
        # FP32 plan's rows and <C, X> in FP32 runs: near 1e-7 the primal
        # residual and the gap are of the size of that rounding)
        k = oracle.kkt(Co, ins.f, ins.g, _np(a.X), _np(a.p), _np(a.q))
        assert abs(k.rel_kkt - a.result["rel_kkt"]) <= 0.1 * tol
        assert k.rel_kkt <= 1.05 * tol
        # the two kernels differ in summation order only: same optimum to the tolerance
        assert abs(a.result["primal_obj"] - b.result["primal_obj"]) / opt < 2 * bound
    r1.close()
    r0.close()


def test_resident_fit_rule():
    """A plan that fits a cluster runs resident (tile_rows 0); one that does
    not runs in tiles."""
    s = pdot.Solver(device=0, time_limit_s=60.0, max_iter=64, resident=1)
    big = (700, 700)
    assert pdot.pdot_resident_fits(*big) == 0
    for (m, n), resident in [((200, 200), True), (big, False)]:
        ins = I.points_instance(m, n, 3500 + m)
        sol = s.solve(torch.tensor(ins.C, dtype=torch.float32, device=DEV), ins.f, ins.g, tol=1e-9)
        assert sol.status == pdot.MAX_ITER
        assert (sol.result["tile_rows"] == 0) == resident
    s.close()


def test_resident_solve_is_deterministic_and_resumable():
    ins = I.points_instance(150, 170, 3600)
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    s = pdot.Solver(device=0, time_limit_s=120.0, resident=1)
    a = s.solve(C, ins.f, ins.g, tol=1e-6)
    b = s.solve(C, ins.f, ins.g, tol=1e-6)
    assert a.result["passes"] == b.result["passes"] and torch.equal(a.X, b.X) and torch.equal(a.p, b.p)
    budget = max(64, (a.result["passes"] // 128) * 64)
    s1 = pdot.Solver(device=0, max_iter=budget, resident=1)
    blob = torch.empty(s1.state_bytes(150, 170), dtype=torch.uint8, device=DEV)
    part = s1.solve(C, ins.f, ins.g, tol=1e-6, state_out=blob)
    assert part.status == pdot.MAX_ITER
    rest = s.solve(C, ins.f, ins.g, tol=1e-6, state_in=blob)
    assert rest.result["passes"] == a.result["passes"] and torch.equal(rest.X, a.X) and torch.equal(rest.q, a.q)
    s.close()
    s1.close()


def test_resident_and_tile_instances_mixed_in_a_batch():
    """Resident instances and tile instances (one too large to fit, one with a
    BF16 cost) in one batch: each result equals the same request alone."""
    reqs = []
    for k, (m, n) in enumerate([(64, 64), (300, 517), (700, 700), (5, 900), (150, 120)]):
        ins = I.points_instance(m, n, 3700 + k, marginals="dirichlet")
        dt = torch.bfloat16 if k == 4 else torch.float32
        reqs.append((torch.tensor(ins.C, dtype=dt, device=DEV), ins.f, ins.g))
    mix = pdot.BatchSolver(device=0, time_limit_s=120.0, resident=1)
    ids = [mix.submit(C, f, g, tol=1e-6) for C, f, g in reqs]
    rm = mix.run()
    mix.close()
    heights = [rm[t].result["tile_rows"] for t in ids]
    assert heights[2] > 0 and heights[0] == 0 and heights[4] == 0
    for tid, (C, f, g) in zip(ids, reqs):
        alone = pdot.BatchSolver(device=0, time_limit_s=120.0, resident=1)
        t2 = alone.submit(C, f, g, tol=1e-6)
        ra = alone.run()[t2]
        alone.close()
        a, b = rm[tid], ra
        assert a.status == b.status == pdot.OK
        assert a.result["passes"] == b.result["passes"] and a.result["primal_obj"] == b.result["primal_obj"]
        assert torch.equal(a.X, b.X) and torch.equal(a.p, b.p) and torch.equal(a.q, b.q)
