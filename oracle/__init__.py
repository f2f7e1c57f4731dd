"""FP64 CPU oracle for PDOT (restarted PDHG for optimal transport, arXiv 2407.19689).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2407_19689_gb300``) never does, and this package never imports it.

Thin ctypes wrapper over ``pdot_oracle.c`` (plain C, FP64, single thread).
Each wrapper names the passage of the paper its C function follows:

- ``apply_A`` / ``apply_At``: Eq. (4) and the implicit products of Sec. 3.1.
- ``pdhg_step``: one inner iteration of Algorithm 2.
- ``lp_pdhg_step``: one inner iteration of Algorithm 1 with an explicit A.
- ``kkt``: the OT KKT error of Sec. 3.1 plus the relative measures (reading C5).
- ``solve``: Algorithm 2 with the Sec. 5 enhancements (or the theory mode).
- ``round_plan``: Algorithm 3.
- ``exact_transport``: the exact optimum of Eq. (1) (successive shortest paths).
- ``dual_bound``: the weak-duality lower bound of Eq. (1) from a row dual p
  (q_j = min_i (C_ij - p_i)).

Parity status: the operators, the PDHG step, the KKT error, the rounding,
the exact solver and the weak-duality bound are pinned by the
``-m "not gpu"`` tests (closed forms, brute force, library LP/assignment
solvers, strong duality at the exact duals, invariants).  The adaptive
heuristics inside ``solve`` are pinned by special cases whose outcome follows
from pinned steps (the restart candidate rule, the artificial-restart
schedule, restart conditions (i) and (ii) each alone, the primal weight at
theta = 0 and 1, the default first step), by one-step cases of the PDLP
step-size rule derived by hand on 1 x 1 and 2 x 1 instances (reject, accept
with omega != 1, growth while the plan stands still, the schedule index),
and end to end (the solve reaches the exact optimum).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdot_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``pdot_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.ora_apply_A.argtypes = [i64, i64, d, d, d]
        lib.ora_apply_At.argtypes = [i64, i64, d, d, d]
        lib.ora_pdhg_step.argtypes = [i64, i64, d, d, d, d, d, d, ctypes.c_double, ctypes.c_double, d, d, d]
        lib.ora_lp_pdhg_step.argtypes = [i64, i64, d, d, d, d, d, ctypes.c_double, ctypes.c_double, d, d]
        lib.ora_kkt.argtypes = [i64, i64, d, d, d, d, d, d, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.POINTER(_KKT)]
        lib.ora_solve.argtypes = [i64, i64, d, d, d, ctypes.POINTER(_Opts), d, d, d, ctypes.POINTER(_Res)]
        lib.ora_solve.restype = ctypes.c_int
        lib.ora_round.argtypes = [i64, i64, d, d, d, d]
        lib.ora_exact_transport.argtypes = [i64, i64, d, d, d, d, d, d, d]
        lib.ora_dual_bound.argtypes = [i64, i64, d, d, d, d, d, d]
        lib.ora_points_cost.argtypes = [i64, i64, ctypes.c_int, d, d, ctypes.c_int, ctypes.c_double, d]
        lib.ora_points_cost.restype = ctypes.c_int
        lib.ora_exact_transport.restype = ctypes.c_int
        _lib = lib
    return _lib


class _KKT(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("rp2", "rd2", "cx", "dual", "gap", "kkt", "rel_p", "rel_d", "rel_gap", "rel_kkt")]


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_passes", ctypes.c_int64), ("check_every", ctypes.c_int64),
                ("adaptive_step", ctypes.c_int), ("adaptive_restart", ctypes.c_int),
                ("primal_weight_update", ctypes.c_int), ("beta", ctypes.c_double),
                ("beta_suff", ctypes.c_double), ("beta_nec", ctypes.c_double), ("beta_art", ctypes.c_double),
                ("theta", ctypes.c_double), ("eta0", ctypes.c_double), ("omega0", ctypes.c_double),
                ("R", ctypes.c_double), ("eps_zero", ctypes.c_double), ("rel_mode", ctypes.c_int)]


class _Res(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("primal_obj", ctypes.c_double), ("dual_obj", ctypes.c_double),
                ("gap", ctypes.c_double), ("kkt", ctypes.c_double), ("rel_p", ctypes.c_double),
                ("rel_d", ctypes.c_double), ("rel_gap", ctypes.c_double), ("rel_kkt", ctypes.c_double),
                ("iters", ctypes.c_int64), ("passes", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("eta", ctypes.c_double), ("omega", ctypes.c_double),
                ("candidate_is_average", ctypes.c_int)]


STATUS_OK = 0
STATUS_MAX_ITER = 5


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def apply_A(X):
    """Eq. (4): returns (X 1_n, X^T 1_m)."""
    X = _f64(X)
    m, n = X.shape
    r, c = np.empty(m), np.empty(n)
    _load().ora_apply_A(m, n, _p(X), _p(r), _p(c))
    return r, c


def apply_At(p, q):
    """Eq. (4): returns p 1_n^T + 1_m q^T."""
    p, q = _f64(p), _f64(q)
    Y = np.empty((p.size, q.size))
    _load().ora_apply_At(p.size, q.size, _p(p), _p(q), _p(Y))
    return Y


def pdhg_step(C, f, g, X, p, q, tau, sigma):
    """One inner iteration of Algorithm 2; returns (X+, p+, q+)."""
    C, f, g, X, p, q = map(_f64, (C, f, g, X, p, q))
    m, n = C.shape
    Xn, pn, qn = np.empty((m, n)), np.empty(m), np.empty(n)
    _load().ora_pdhg_step(m, n, _p(C), _p(f), _p(g), _p(X), _p(p), _p(q), float(tau), float(sigma),
                          _p(Xn), _p(pn), _p(qn))
    return Xn, pn, qn


def pdhg_steps(C, f, g, X, p, q, k, eta, omega=1.0):
    """k inner iterations of Algorithm 2 at constant (eta, omega), with the
    uniform running average; returns (X, p, q, Xbar, pbar, qbar)."""
    X, p, q = _f64(X), _f64(p), _f64(q)
    Xb, pb, qb = X.copy(), p.copy(), q.copy()
    tau, sigma = eta / omega, eta * omega
    for j in range(k):
        X, p, q = pdhg_step(C, f, g, X, p, q, tau, sigma)
        if j == 0:
            Xb, pb, qb = X.copy(), p.copy(), q.copy()
        else:
            wo, wn = j / (j + 1.0), 1.0 / (j + 1.0)
            Xb, pb, qb = wo * Xb + wn * X, wo * pb + wn * p, wo * qb + wn * q
    return X, p, q, Xb, pb, qb


def lp_pdhg_step(A, b, c, x, y, eta, sigma):
    """One inner iteration of Algorithm 1 on min c^T x s.t. Ax=b, x>=0 (explicit A)."""
    A, b, c, x, y = map(_f64, (A, b, c, x, y))
    M, N = A.shape
    xn, yn = np.empty(N), np.empty(M)
    _load().ora_lp_pdhg_step(M, N, _p(A), _p(b), _p(c), _p(x), _p(y), float(eta), float(sigma), _p(xn), _p(yn))
    return xn, yn


@dataclass
class KKT:
    rp2: float
    rd2: float
    cx: float
    dual: float
    gap: float
    kkt: float
    rel_p: float
    rel_d: float
    rel_gap: float
    rel_kkt: float


def kkt(C, f, g, X, p, q, R=1.0, rel_mode=0):
    """KKT error of Sec. 3.1 and the relative measures of reading C5."""
    C, f, g, X, p, q = map(_f64, (C, f, g, X, p, q))
    m, n = C.shape
    nb = float(np.sqrt(np.sum(f * f) + np.sum(g * g)))
    nc = float(np.sqrt(np.sum(C * C)))
    out = _KKT()
    _load().ora_kkt(m, n, _p(C), _p(f), _p(g), _p(X), _p(p), _p(q), float(R), nb, nc, int(rel_mode),
                    ctypes.byref(out))
    return KKT(*[getattr(out, k) for k, _ in _KKT._fields_])


@dataclass
class Options:
    tol: float = 1e-6
    max_passes: int = 1_000_000
    check_every: int = 64
    adaptive_step: int = 1
    adaptive_restart: int = 1
    primal_weight_update: int = 1
    beta: float = 0.2
    beta_suff: float = 0.1
    beta_nec: float = 0.9
    beta_art: float = 0.36
    theta: float = 0.5
    eta0: float = 0.0
    omega0: float = 1.0
    R: float = 1.0
    eps_zero: float = 1e-10
    rel_mode: int = 0


@dataclass
class Result:
    status: int
    primal_obj: float
    dual_obj: float
    gap: float
    kkt: float
    rel_p: float
    rel_d: float
    rel_gap: float
    rel_kkt: float
    iters: int
    passes: int
    restarts: int
    rejected: int
    eta: float
    omega: float
    candidate_is_average: int
    X: np.ndarray = None
    p: np.ndarray = None
    q: np.ndarray = None


def solve(C, f, g, opts: Options | None = None, X0=None, p0=None, q0=None) -> Result:
    """Algorithm 2 + Sec. 5 in FP64.  Default start X=0, p=0, q=0 (reading C1)."""
    opts = opts or Options()
    C, f, g = map(_f64, (C, f, g))
    m, n = C.shape
    X = np.zeros((m, n)) if X0 is None else _f64(X0).copy()
    p = np.zeros(m) if p0 is None else _f64(p0).copy()
    q = np.zeros(n) if q0 is None else _f64(q0).copy()
    o = _Opts(**{k: getattr(opts, k) for k, _ in _Opts._fields_})
    r = _Res()
    _load().ora_solve(m, n, _p(C), _p(f), _p(g), ctypes.byref(o), _p(X), _p(p), _p(q), ctypes.byref(r))
    res = Result(*[getattr(r, k) for k, _ in _Res._fields_])
    res.X, res.p, res.q = X, p, q
    return res


def round_plan(X, f, g):
    """Algorithm 3: an exactly feasible plan near X."""
    X, f, g = map(_f64, (X, f, g))
    m, n = X.shape
    Xf = np.empty((m, n))
    _load().ora_round(m, n, _p(X), _p(f), _p(g), _p(Xf))
    return Xf


def exact_transport(C, f, g):
    """Exact optimum of Eq. (1); returns (objective, X, p, q)."""
    C, f, g = map(_f64, (C, f, g))
    m, n = C.shape
    X, p, q = np.empty((m, n)), np.empty(m), np.empty(n)
    obj = ctypes.c_double()
    rc = _load().ora_exact_transport(m, n, _p(C), _p(f), _p(g), _p(X), _p(p), _p(q), ctypes.byref(obj))
    if rc != 0:
        raise RuntimeError(f"exact_transport failed (code {rc})")
    return obj.value, X, p, q


def dual_bound(C, f, g, p):
    """Weak duality of Eq. (1): q_j = min_i (C_ij - p_i) is the largest column
    dual feasible with p, and f^T p + g^T q <= OPT.  Returns (lower, q)."""
    C, f, g, p = map(_f64, (C, f, g, p))
    m, n = C.shape
    q = np.empty(n)
    lower = np.empty(1)
    _load().ora_dual_bound(m, n, _p(C), _p(f), _p(g), _p(p), _p(q), _p(lower))
    return float(lower[0]), q


POINT_DISTANCES = {"sqeuclid": 0, "l1": 1, "l2": 2, "linf": 3}


def points_cost(xs, ys, dist: str = "sqeuclid", divisor: float = 1.0):
    """C_ij = dist(xs_i, ys_j) / divisor in FP64 (the cost-on-the-fly input)."""
    xs, ys = _f64(np.atleast_2d(xs)), _f64(np.atleast_2d(ys))
    m, d = xs.shape
    n = ys.shape[0]
    assert ys.shape[1] == d
    C = np.empty((m, n))
    rc = _load().ora_points_cost(m, n, d, _p(xs), _p(ys), POINT_DISTANCES[dist], float(divisor), _p(C))
    if rc != 0:
        raise ValueError("points_cost: bad arguments")
    return C
