"""Warm start and checkpoint / resume (pdot_solve_from), on the GPU.

- A solve stopped by its pass budget, or by its time limit, and resumed from
  the exported state takes the same passes and returns the same result, bit
  for bit, as the uninterrupted solve.
- Started at the exact optimum (oracle's exact transportation solver), a solve
  stops at its initial check with the optimal objective.
- The one-pass step-size cases derived by hand (tests/heuristic_cases.py),
  which start away from the origin, give the derived counts, step size and
  point on the GPU (FP64 plans).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from heuristic_cases import STEP_RULE_CASES  # noqa: E402
from paper_2407_19689_gb300 import instances as I  # noqa: E402
from paper_2407_19689_gb300 import pdot  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    pdot.load(build_if_missing=True)


def _blob(s, m, n):
    return torch.empty(s.state_bytes(m, n), dtype=torch.uint8, device=DEV)


def _same(a, b):
    ra, rb = a.result, b.result
    for key in ("passes", "iters", "restarts", "rejected_steps", "primal_obj", "rel_kkt", "eta", "omega"):
        assert ra[key] == rb[key], (key, ra[key], rb[key])
    assert torch.equal(a.X, b.X) and torch.equal(a.p, b.p) and torch.equal(a.q, b.q)


@pytest.mark.parametrize("xt", [pdot.F32, pdot.F64])
def test_resume_after_pass_budget_equals_uninterrupted(xt):
    ins = I.points_instance(300, 517, 91, marginals="dirichlet")
    dt = torch.float32 if xt == pdot.F32 else torch.float64
    C = torch.tensor(ins.C, dtype=dt, device=DEV)
    full = pdot.Solver(device=0, x_dtype=xt, time_limit_s=120.0).solve(C, ins.f, ins.g, tol=1e-6)
    assert full.status == pdot.OK
    P = full.result["passes"]
    budget = max(64, (P // 128) * 64)   # a check about halfway
    s1 = pdot.Solver(device=0, x_dtype=xt, max_iter=budget)
    blob = _blob(s1, 300, 517)
    part = s1.solve(C, ins.f, ins.g, tol=1e-6, state_out=blob)
    assert part.status == pdot.MAX_ITER and part.result["passes"] == budget
    # resume on another handle (same options, same kernel choice for this shape)
    s2 = pdot.Solver(device=0, x_dtype=xt, time_limit_s=120.0)
    rest = s2.solve(C, ins.f, ins.g, tol=1e-6, state_in=blob)
    assert rest.status == pdot.OK
    _same(rest, full)
    # a three-way split: stop again, resume again
    s3 = pdot.Solver(device=0, x_dtype=xt, max_iter=budget + 64)
    blob2 = _blob(s3, 300, 517)
    mid = s3.solve(C, ins.f, ins.g, tol=1e-6, state_in=blob, state_out=blob2)
    assert mid.status == pdot.MAX_ITER and mid.result["passes"] == budget + 64
    _same(s2.solve(C, ins.f, ins.g, tol=1e-6, state_in=blob2), full)
    for s in (s1, s2, s3):
        s.close()


def test_resume_after_time_limit_equals_uninterrupted():
    ins = I.points_instance(257, 300, 92)
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    full = pdot.Solver(device=0, time_limit_s=120.0).solve(C, ins.f, ins.g, tol=1e-6)
    s1 = pdot.Solver(device=0, time_limit_s=1e-9)
    blob = _blob(s1, 257, 300)
    part = s1.solve(C, ins.f, ins.g, tol=1e-6, state_out=blob)
    assert part.status == pdot.TIMEOUT and 0 < part.result["passes"] < full.result["passes"]
    s2 = pdot.Solver(device=0, time_limit_s=120.0)
    _same(s2.solve(C, ins.f, ins.g, tol=1e-6, state_in=blob), full)
    s1.close()
    s2.close()


def test_state_of_another_shape_is_rejected():
    ins = I.points_instance(40, 50, 93)
    C = torch.tensor(ins.C, dtype=torch.float32, device=DEV)
    s = pdot.Solver(device=0, max_iter=64)
    blob = _blob(s, 40, 50)
    s.solve(C, ins.f, ins.g, tol=1e-6, state_out=blob)
    ins2 = I.points_instance(50, 40, 94)
    big = torch.zeros(s.state_bytes(50, 40) + 4096, dtype=torch.uint8, device=DEV)
    big[: blob.numel()] = blob
    with pytest.raises(pdot.PdotError) as e:
        s.solve(torch.tensor(ins2.C, dtype=torch.float32, device=DEV), ins2.f, ins2.g, tol=1e-6, state_in=big)
    assert e.value.status == pdot.ERR_ARG
    zeros = torch.zeros_like(blob)
    with pytest.raises(pdot.PdotError) as e:
        s.solve(C, ins.f, ins.g, tol=1e-6, state_in=zeros)
    assert e.value.status == pdot.ERR_ARG
    s.close()


def test_warm_start_at_the_exact_optimum_stops_at_once():
    """Started at an exact optimum (X*, p*, q*) of Eq. (1), the KKT error is 0
    up to rounding: the initial check terminates with no pass."""
    ins = I.points_instance(60, 45, 95)
    opt, Xs, ps, qs = oracle.exact_transport(ins.C, ins.f, ins.g)
    s = pdot.Solver(device=0, x_dtype=pdot.F64, time_limit_s=60.0)
    sol = s.solve(torch.tensor(ins.C, device=DEV), ins.f, ins.g, tol=1e-9, X0=Xs, p0=ps, q0=qs)
    s.close()
    assert sol.status == pdot.OK and sol.result["passes"] == 0
    assert abs(sol.result["primal_obj"] - opt) <= 1e-12 * opt
    assert np.array_equal(sol.X.cpu().numpy(), Xs)


@pytest.mark.parametrize("case", STEP_RULE_CASES, ids=lambda c: c["name"])
def test_step_rule_one_pass_by_hand_on_gpu(case):
    """The one-pass step-size cases derived by hand, started at their given
    points through pdot_solve_from (FP64 plans, a check after the pass)."""
    s = pdot.Solver(device=0, x_dtype=pdot.F64, restart_check_every=1, max_iter=1, eta0=case["eta0"],
                    omega0=case["omega0"], primal_weight_update=0, time_limit_s=60.0)
    C = torch.tensor(case["C"], dtype=torch.float64, device=DEV)
    sol = s.solve(C, np.array(case["f"]), np.array(case["g"]), tol=1e-15, X0=np.array(case["X0"]),
                  p0=np.array(case["p0"]), q0=np.array(case["q0"]))
    s.close()
    r = sol.result
    assert sol.status == pdot.MAX_ITER
    assert (r["passes"], r["iters"], r["rejected_steps"]) == (1, case["iters"], case["rejected"])
    assert abs(r["eta"] - case["eta"]) <= 1e-15
    assert np.array_equal(sol.X.cpu().numpy(), np.array(case["X"]))
    assert np.array_equal(sol.p.cpu().numpy(), np.array(case["p"]))
    assert np.array_equal(sol.q.cpu().numpy(), np.array(case["q"]))
