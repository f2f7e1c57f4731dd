"""Certified lower bound on the optimum of Eq. (1) from a row dual
(pdot_dual_bound): q_j = min_i (C_ij - p_i) and f^T p + g^T q <= OPT.

- parity with the FP64 oracle (oracle.dual_bound) on the same cost values:
  q bit for bit (a minimum is exact), the bound to the rounding of its two
  dot products, for FP32, BF16 and FP64 stored costs and the cost generated
  from pixel-grid coordinates, on shapes with ragged column blocks, fewer
  rows than row groups and more;
- with the duals of GPU solves (single and batched) and the Algorithm 3
  rounding of their plans, the interval [bound, rounded objective] contains
  the exact optimum;
- argument errors.
"""
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


def _check(lower, q, C64, f, g, p):
    lo, qo = oracle.dual_bound(C64, f, g, p)
    np.testing.assert_array_equal(_np(q), qo)
    scale = np.abs(f * p).sum() + np.abs(g * qo).sum()
    assert abs(lower - lo) <= 1e-13 * scale, (lower, lo)


@pytest.mark.parametrize("m,n", [(1, 7), (37, 53), (130, 517), (300, 80), (1000, 33)])
@pytest.mark.parametrize("cdt", ["f32", "bf16", "f64"])
def test_dual_bound_matches_oracle(m, n, cdt):
    ins = I.points_instance(m, n, 4000 + m + n)
    rng = np.random.default_rng(m * 7 + n)
    p = rng.standard_normal(m) * 0.1
    if cdt == "f64":
        s = pdot.Solver(device=0, x_dtype=pdot.F64)
        Cd = torch.tensor(ins.C, dtype=torch.float64, device=DEV)
    else:
        s = pdot.Solver(device=0)
        Cd = torch.tensor(ins.C, dtype=torch.float32 if cdt == "f32" else torch.bfloat16, device=DEV)
    lower, q = s.dual_bound(Cd, ins.f, ins.g, p)
    _check(lower, q, _np(Cd), ins.f, ins.g, p)
    s.close()


def test_dual_bound_strided_cost():
    """A cost with a leading dimension larger than n (ldc = 128, n = 90),
    through the C entry point."""
    ins = I.points_instance(70, 90, 4100)
    big = torch.zeros((70, 128), dtype=torch.float32, device=DEV)
    big[:, :90] = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    p = np.random.default_rng(5).standard_normal(70) * 0.1
    pd = torch.tensor(p, device=DEV)
    f = torch.tensor(ins.f, device=DEV)
    g = torch.tensor(ins.g, device=DEV)
    q = torch.empty(90, dtype=torch.float64, device=DEV)
    s = pdot.Solver(device=0)
    st, lower = pdot.pdot_dual_bound(s.h, 70, 90, big.data_ptr(), pdot.F32, 128, f.data_ptr(), g.data_ptr(),
                                     pd.data_ptr(), q.data_ptr())
    assert st == pdot.OK
    _check(lower, q, _np(big[:, :90]), ins.f, ins.g, p)
    s.close()


@pytest.mark.parametrize("G", [8, 23])
def test_dual_bound_generated_cost_on_a_pixel_grid(G):
    """Cost generated from pixel coordinates: on an integer grid the FP32
    value is the correctly rounded stored cost, so the oracle takes the
    stored FP32 matrix."""
    ins = I.grid_blob_instance(G, I.seed_for(1, 3))
    P = I.grid_coords(G).astype(np.float32)
    div = float(2 * (G - 1) ** 2)
    p = np.random.default_rng(G).standard_normal(G * G) * 0.05
    s = pdot.Solver(device=0)
    lower, q = s.dual_bound(pdot.Points(P, P, "sqeuclid", div), ins.f, ins.g, p)
    _check(lower, q, ins.C.astype(np.float32).astype(np.float64), ins.f, ins.g, p)
    s.close()


@pytest.mark.parametrize("m,n,seed", [(64, 64, I.seed_for(0)), (37, 51, 101), (120, 45, 4200)])
def test_solve_optimum_lies_in_the_certified_interval(m, n, seed):
    """A GPU solve's duals give a bound below the exact optimum, and the
    Algorithm 3 rounding of its plan (FP64, so exactly feasible up to FP64
    rounding) an objective above it."""
    ins = I.points_instance(m, n, seed)
    opt, *_ = oracle.exact_transport(ins.C, ins.f, ins.g)
    s = pdot.Solver(device=0, x_dtype=pdot.F64, round_plan=1, time_limit_s=120.0)
    Cd = torch.tensor(ins.C, dtype=torch.float64, device=DEV)
    sol = s.solve(Cd, ins.f, ins.g, tol=1e-6)
    assert sol.status == pdot.OK
    lower, q = s.dual_bound(Cd, ins.f, ins.g, sol.p)
    _check(lower, q, ins.C, ins.f, ins.g, _np(sol.p))
    upper = sol.result["rounded_obj"]
    assert lower <= opt + 1e-14 * opt and opt <= upper + 1e-14 * opt, (lower, opt, upper)
    assert (upper - lower) / lower < 1e-3
    s.close()


def test_batched_results_are_certified():
    """Each batched result's duals bound the optimum of its own instance from
    below."""
    insts = [I.points_instance(m, n, 4300 + k) for k, (m, n) in enumerate([(40, 60), (90, 33), (17, 128)])]
    b = pdot.BatchSolver(device=0, time_limit_s=120.0)
    tick = {}
    for ins in insts:
        Cd = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
        tick[b.submit(Cd, ins.f, ins.g, tol=1e-6)] = (ins, Cd)
    done = b.run()
    b.close()
    s = pdot.Solver(device=0)
    for t, sol in done.items():
        ins, Cd = tick[t]
        assert sol.status == pdot.OK
        opt, *_ = oracle.exact_transport(_np(Cd), ins.f, ins.g)
        lower, q = s.dual_bound(Cd, ins.f, ins.g, sol.p)
        _check(lower, q, _np(Cd), ins.f, ins.g, _np(sol.p))
        assert lower <= opt * (1 + 1e-12)
        assert (opt - lower) / opt < 1e-3
    s.close()


def test_dual_bound_argument_errors():
    ins = I.points_instance(5, 6, 4400)
    s = pdot.Solver(device=0)
    Cd = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    f = torch.tensor(ins.f, device=DEV)
    g = torch.tensor(ins.g, device=DEV)
    p = torch.zeros(5, dtype=torch.float64, device=DEV)
    st, _ = pdot.pdot_dual_bound(s.h, 5, 6, Cd.data_ptr(), pdot.F32, 6, f.data_ptr(), g.data_ptr(), 0)
    assert st == pdot.ERR_ARG
    st, _ = pdot.pdot_dual_bound(s.h, 5, 6, Cd.data_ptr(), pdot.F32, 5, f.data_ptr(), g.data_ptr(), p.data_ptr())
    assert st == pdot.ERR_ARG   # ldc < n
    C64 = Cd.double()
    st, _ = pdot.pdot_dual_bound(s.h, 5, 6, C64.data_ptr(), pdot.F64, 6, f.data_ptr(), g.data_ptr(), p.data_ptr())
    assert st == pdot.ERR_ARG   # FP64 cost on a handle with FP32 plans
    st, lower = pdot.pdot_dual_bound(s.h, 5, 6, Cd.data_ptr(), pdot.F32, 6, f.data_ptr(), g.data_ptr(),
                                     p.data_ptr())
    assert st == pdot.OK and abs(lower - float(ins.g @ _np(Cd).min(axis=0))) <= 1e-15
    s.close()
