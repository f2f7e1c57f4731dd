"""The allocation-free rounding entry point (pdot_round_noalloc).

It exists for callers that cannot allocate device memory when they round a
plan (memory owned by another allocator, serving loops that forbid
cudaMalloc after warm-up, plug-ins inside applications that own every
allocation).  Checked through the C ABI against the allocating pdot_round and
against the FP64 oracle's Algorithm 3, on two calls in a row (the static
scratch array is reused by the second call), in place (X_out = X), and from
two host threads on two streams at once (the library runs them one after the
other).  This file is collected last on purpose.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2407_19689_gb300 import pdot  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    pdot.load(build_if_missing=True)


def _case(m, n, seed, dt):
    rng = np.random.default_rng(seed)
    f, g = rng.dirichlet(np.ones(m)), rng.dirichlet(np.ones(n))
    X = torch.tensor(np.outer(f, g) * rng.uniform(0.5, 1.5, (m, n)), dtype=dt, device=DEV)
    return X, f, g, torch.tensor(f, device=DEV), torch.tensor(g, device=DEV)


def _rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = b.double().cpu().numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _call(stream, m, n, xt, X, fd, gd, out):
    return pdot.pdot_round_noalloc(0, stream, m, n, xt, X.data_ptr(), fd.data_ptr(), gd.data_ptr(), out.data_ptr())


@pytest.mark.parametrize("xt", [pdot.F64, pdot.F32])
def test_round_noalloc_matches_round_and_oracle_twice(xt):
    dt = torch.float64 if xt == pdot.F64 else torch.float32
    tol = 1e-13 if xt == pdot.F64 else 1e-6
    ref = pdot.Solver(device=0, x_dtype=xt)
    for m, n in [(300, 517), (129, 33)]:
        X, f, g, fd, gd = _case(m, n, 11 + m, dt)
        want = ref.round(X, f, g)
        got = torch.empty_like(X)
        assert _call(torch.cuda.current_stream().cuda_stream, m, n, xt, X, fd, gd, got) == pdot.OK
        assert _rel(got, want) < tol
        assert _rel(got, oracle.round_plan(X.double().cpu().numpy(), f, g)) < tol
        if xt == pdot.F64:
            np.testing.assert_allclose(got.sum(1).cpu().numpy(), f, atol=1e-15)
            np.testing.assert_allclose(got.sum(0).cpu().numpy(), g, atol=1e-15)
    ref.close()


def test_round_noalloc_in_place():
    """X_out may alias X: each output entry is written by the thread that read
    it, after every sum that needs X is complete."""
    ref = pdot.Solver(device=0, x_dtype=pdot.F64)
    m, n = 257, 190
    X, f, g, fd, gd = _case(m, n, 41, torch.float64)
    want = ref.round(X, f, g)
    Y = X.clone()
    assert _call(torch.cuda.current_stream().cuda_stream, m, n, pdot.F64, Y, fd, gd, Y) == pdot.OK
    assert _rel(Y, want) < 1e-13
    ref.close()


def test_round_noalloc_two_threads_two_streams():
    """Two host threads, each on its own stream with its own shape, call at
    the same time; the library lets one call use the shared scratch at a
    time, so both results equal pdot_round's."""
    ref = pdot.Solver(device=0, x_dtype=pdot.F64)
    cases = [(_case(400, 350, 51, torch.float64), (400, 350)), (_case(90, 1200, 52, torch.float64), (90, 1200))]
    outs = [torch.empty_like(c[0][0]) for c in cases]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    status = [None, None]
    start = threading.Barrier(2)

    def work(k):
        (X, f, g, fd, gd), (m, n) = cases[k]
        start.wait()
        for _ in range(3):
            status[k] = _call(streams[k].cuda_stream, m, n, pdot.F64, X, fd, gd, outs[k])
            if status[k] != pdot.OK:
                return

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert status == [pdot.OK, pdot.OK]
    for k, ((X, f, g, _, _), _) in enumerate(cases):
        assert _rel(outs[k], ref.round(X, f, g)) < 1e-13
    ref.close()


def test_round_noalloc_rejects_sizes_beyond_its_array():
    assert pdot.pdot_round_noalloc(0, 0, 40000, 10, pdot.F32, 1, 1, 1, 1) == pdot.ERR_ARG
    assert pdot.pdot_round_noalloc(0, 0, 10, 0, pdot.F32, 1, 1, 1, 1) == pdot.ERR_ARG
