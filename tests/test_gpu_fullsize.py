"""Full-size single-instance shapes on the GPU, checked where the oracle can:

- 16384 x 16384 (128 x 128 grid, blob marginals), FP32 and BF16 costs;
- 8192 x 32768 rectangular, L1 cost between uniform points in [0,1]^3 (/3).

One PDHG step from an iterate the GPU produced is checked row by row on a
sample of rows against the oracle's step on those rows (the primal update and
p+ are row-local), and q+ against the dual update applied to the full column
sums of the returned plans (a property that holds at any size).
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


def _grid128_device():
    ins = I.grid_blob_instance(128, I.seed_for(2), build_cost=False)
    P = torch.tensor(I.grid_coords(128), device=DEV)
    C = torch.cdist(P, P) ** 2
    C /= C.max()
    return C, ins.f, ins.g


def _rect_device():
    rng = np.random.default_rng(I.seed_for(2, 1))
    xs, ys = rng.random((8192, 3)), rng.random((32768, 3))
    f = rng.dirichlet(np.ones(8192))
    g = rng.dirichlet(np.ones(32768))
    f, g = f / f.sum(), g / g.sum()
    C = torch.cdist(torch.tensor(xs, device=DEV), torch.tensor(ys, device=DEV), p=1.0) / 3.0
    return C, f, g


def _check_step(C, f, g, dtype, k0=3, rows=48):
    m, n = C.shape
    Cd = C.to(dtype)
    s = pdot.Solver(device=0)
    eta = 0.7 / math.sqrt(m + n)
    z = (torch.zeros((m, n), device=DEV), torch.zeros(m, dtype=torch.float64, device=DEV),
         torch.zeros(n, dtype=torch.float64, device=DEV))
    X2, p2, q2, *_ = s.pdhg_steps(Cd, f, g, *z, k=k0, eta=eta)
    X3, p3, q3, *_ = s.pdhg_steps(Cd, f, g, X2, p2, q2, k=1, eta=eta)
    rng = np.random.default_rng(5)
    S = np.sort(rng.choice(m, rows, replace=False))
    St = torch.tensor(S, device=DEV)
    Cs = Cd.index_select(0, St).double().cpu().numpy()
    X2s = X2.index_select(0, St).double().cpu().numpy()
    q2h = q2.cpu().numpy()
    p2s = p2.index_select(0, St).cpu().numpy()
    # the oracle's step on the sampled rows (g only enters q+, not compared here)
    Xo, po, _ = oracle.pdhg_step(Cs, f[S], np.full(n, 1.0 / n) * f[S].sum(), X2s, p2s, q2h, eta, eta)
    X3s = X3.index_select(0, St).double().cpu().numpy()
    assert np.linalg.norm(X3s - Xo) <= 1e-5 * np.linalg.norm(Xo) + 1e-12
    np.testing.assert_allclose(p3.index_select(0, St).cpu().numpy(), po, rtol=1e-5, atol=1e-12)
    # q+ = q + sigma (g - (2 c+ - c)) with the full column sums of the plans
    c2 = X2.double().sum(0)
    c3 = X3.double().sum(0)
    q_expect = q2 + eta * (torch.tensor(g, device=DEV) - (2.0 * c3 - c2))
    err = (torch.linalg.norm(q3 - q_expect) / torch.linalg.norm(q_expect)).item()
    assert err < 1e-5, err
    s.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_grid128_step(dtype):
    C, f, g = _grid128_device()
    _check_step(C, f, g, torch.float32 if dtype == "f32" else torch.bfloat16)


def test_rect_8192x32768_l1_step():
    C, f, g = _rect_device()
    _check_step(C, f, g, torch.float32)
