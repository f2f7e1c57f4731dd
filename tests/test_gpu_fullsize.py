"""Full-size single-instance shapes on the GPU, every plan-pass kernel, checked
against the FP64 oracle where it can run:

- 4096 x 4096 (64 x 64 grid, blob marginals), FP32 and BF16 costs: 100 PDHG
  steps (Algorithm 2) of each pass kernel against the oracle's 100 steps, every
  element of X, p, q and of the running averages compared;
- 16384 x 16384 (128 x 128 grid), FP32 and BF16 costs, and the rectangular
  8192 x 32768 L1 case: one PDHG step from an iterate the GPU produced,
  checked against the oracle's step on a sample of rows (the primal update
  and p+ are row-local) and on a sample of columns (q+ needs only its
  column's full sums of X and X+).

Bounds (FP32 plan, FP64 duals; 2^-24 rounding of the plan and of the reduced
cost per step): relative Frobenius error <= 1e-5 and largest element error
<= 1e-5 of the largest element, for every compared array.
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
# pass_kernel option values: 1 register pipeline, 2 bulk copies per row, 3 bulk copies per 4-row group
KERNELS = {1: "register", 2: "bulk-row", 3: "bulk-group"}
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    pdot.load(build_if_missing=True)


def _np(t):
    return t.double().cpu().numpy()


def _close(got, want, name):
    """Relative Frobenius error and largest element error, both <= TOL."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = float(np.max(np.abs(want)))
    nw = float(np.linalg.norm(want))
    fro = float(np.linalg.norm(got - want)) / (nw if nw > 0 else 1.0)
    mx = float(np.max(np.abs(got - want))) / (scale if scale > 0 else 1.0)
    assert fro <= TOL and mx <= TOL, (name, fro, mx)
    return fro, mx


def _grid_cost_device(G):
    P = torch.tensor(I.grid_coords(G), device=DEV)
    C = torch.cdist(P, P) ** 2
    return C / C.max()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_grid64_100_steps_every_kernel(dtype):
    """4096^2: 100 constant-step iterations from X = 0, p = q = 0.05 (the
    reduced cost C - p - q is negative on about half of the entries, so the
    plan is dense at first) by each pass kernel, against the oracle."""
    ins = I.grid_blob_instance(64, I.seed_for(1), build_cost=False)
    C = _grid_cost_device(64).to(torch.float32 if dtype == "f32" else torch.bfloat16)
    m = n = 4096
    Co = _np(C)
    X0, p0, q0 = np.zeros((m, n)), np.full(m, 0.05), np.full(n, 0.05)
    eta = 0.7 / math.sqrt(m + n)
    k = 100
    want = oracle.pdhg_steps(Co, ins.f, ins.g, X0, p0, q0, k=k, eta=eta, omega=1.0)
    del Co
    assert np.count_nonzero(want[3]) > m * n // 10   # the average keeps the dense early plans
    for kern in KERNELS:
        s = pdot.Solver(device=0, pass_kernel=kern)
        got = s.pdhg_steps(C, ins.f, ins.g, X0, p0, q0, k=k, eta=eta, omega=1.0)
        s.close()
        for a, b, name in zip(got, want, ("X", "p", "q", "Xbar", "pbar", "qbar")):
            _close(_np(a), b, f"{KERNELS[kern]} {dtype} {name}")
        del got
        torch.cuda.empty_cache()


def _check_step(C, f, g, kern, k0=3, rows=48, cols=48):
    m, n = C.shape
    s = pdot.Solver(device=0, pass_kernel=kern)
    eta = 0.7 / math.sqrt(m + n)
    z = (torch.zeros((m, n), device=DEV), torch.zeros(m, dtype=torch.float64, device=DEV),
         torch.zeros(n, dtype=torch.float64, device=DEV))
    X2, p2, q2, *_ = s.pdhg_steps(C, f, g, *z, k=k0, eta=eta)
    X3, p3, q3, *_ = s.pdhg_steps(C, f, g, X2, p2, q2, k=1, eta=eta)
    s.close()
    rng = np.random.default_rng(5)
    # rows: the primal update and p+ of a row need only that row
    S = torch.tensor(np.sort(rng.choice(m, rows, replace=False)), device=DEV)
    Cs = _np(C.index_select(0, S))
    fs = f[S.cpu().numpy()]
    Xo, po, _ = oracle.pdhg_step(Cs, fs, np.full(n, fs.sum() / n), _np(X2.index_select(0, S)),
                                 p2.index_select(0, S).cpu().numpy(), q2.cpu().numpy(), eta, eta)
    _close(_np(X3.index_select(0, S)), Xo, "X+ rows")
    _close(p3.index_select(0, S).cpu().numpy(), po, "p+ rows")
    # columns: q+_j = q_j + sigma (g_j - (2 c+_j - c_j)) needs column j of X and X+ only
    T = torch.tensor(np.sort(rng.choice(n, cols, replace=False)), device=DEV)
    gt = g[T.cpu().numpy()]
    Ct = _np(C.index_select(1, T))
    Xc, _, qo = oracle.pdhg_step(Ct, np.full(m, gt.sum() / m), gt, _np(X2.index_select(1, T)), p2.cpu().numpy(),
                                 q2.index_select(0, T).cpu().numpy(), eta, eta)
    _close(_np(X3.index_select(1, T)), Xc, "X+ columns")
    _close(q3.index_select(0, T).cpu().numpy(), qo, "q+ columns")


@pytest.mark.parametrize("kern", sorted(KERNELS))
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_grid128_step_every_kernel(dtype, kern):
    ins = I.grid_blob_instance(128, I.seed_for(2), build_cost=False)
    C = _grid_cost_device(128).to(torch.float32 if dtype == "f32" else torch.bfloat16)
    _check_step(C, ins.f, ins.g, kern)


@pytest.mark.parametrize("kern", [2, 3])
def test_rect_8192x32768_l1_step(kern):
    rng = np.random.default_rng(I.seed_for(2, 1))
    xs, ys = rng.random((8192, 3)), rng.random((32768, 3))
    f = rng.dirichlet(np.ones(8192))
    g = rng.dirichlet(np.ones(32768))
    f, g = f / f.sum(), g / g.sum()
    C = (torch.cdist(torch.tensor(xs, device=DEV), torch.tensor(ys, device=DEV), p=1.0) / 3.0).float()
    _check_step(C, f, g, kern)
