"""Time limits: a solve past its wall-clock limit returns the current iterate
with that iterate's own KKT measures (status PDOT_TIMEOUT)."""
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


def test_time_limit_returns_the_current_iterate():
    """A solve past its time limit stops at the next chunk boundary and
    reports the current iterate with that iterate's own KKT measures."""
    ins = I.points_instance(300, 517, 81)
    s = pdot.Solver(device=0, time_limit_s=1e-9)
    sol = s.solve(torch.tensor(ins.C, dtype=torch.float32, device=DEV), ins.f, ins.g, tol=1e-9)
    s.close()
    passes = sol.result["passes"]
    assert sol.status == pdot.TIMEOUT and sol.result["returned_average"] == 0
    assert passes > 0 and passes % 64 == 0
    k = oracle.kkt(ins.C.astype(np.float32).astype(np.float64), ins.f, ins.g, _np(sol.X), _np(sol.p), _np(sol.q))
    assert abs(k.rel_kkt - sol.result["rel_kkt"]) <= 1e-4 * k.rel_kkt
