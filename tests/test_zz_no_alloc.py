"""The allocation-free rounding entry point (pdot_round_noalloc).

It exists for callers that cannot allocate device memory when they round a
plan (memory owned by another allocator, serving loops that forbid
cudaMalloc after warm-up, plug-ins inside applications that own every
allocation).  Checked through the C ABI against the allocating pdot_round, on
two calls in a row (the static scratch array is reused by the second call).
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_19689_gb300 import pdot  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("xt", [pdot.F64, pdot.F32])
def test_round_noalloc_matches_round_twice(xt):
    pdot.load(build_if_missing=True)
    dt = torch.float64 if xt == pdot.F64 else torch.float32
    ref = pdot.Solver(device=0, x_dtype=xt)
    rng = np.random.default_rng(11)
    for m, n in [(300, 517), (129, 33)]:
        f, g = rng.dirichlet(np.ones(m)), rng.dirichlet(np.ones(n))
        X = torch.tensor(np.outer(f, g) * rng.uniform(0.5, 1.5, (m, n)), dtype=dt, device=DEV)
        fd = torch.tensor(f, device=DEV)
        gd = torch.tensor(g, device=DEV)
        want = ref.round(X, f, g)
        got = torch.empty_like(X)
        st = pdot.pdot_round_noalloc(0, torch.cuda.current_stream().cuda_stream, m, n, xt, X.data_ptr(),
                                     fd.data_ptr(), gd.data_ptr(), got.data_ptr())
        assert st == pdot.OK
        err = (torch.linalg.norm((got - want).double()) / torch.linalg.norm(want.double())).item()
        assert err < (1e-13 if xt == pdot.F64 else 1e-6), err
        if xt == pdot.F64:
            np.testing.assert_allclose(got.sum(1).cpu().numpy(), f, atol=1e-15)
            np.testing.assert_allclose(got.sum(0).cpu().numpy(), g, atol=1e-15)
    ref.close()


def test_round_noalloc_rejects_sizes_beyond_its_array():
    pdot.load(build_if_missing=True)
    assert pdot.pdot_round_noalloc(0, 0, 40000, 10, pdot.F32, 1, 1, 1, 1) == pdot.ERR_ARG
    assert pdot.pdot_round_noalloc(0, 0, 10, 0, pdot.F32, 1, 1, 1, 1) == pdot.ERR_ARG
