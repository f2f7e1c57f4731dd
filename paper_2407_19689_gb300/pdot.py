"""Python binding of the C ABI in ``include/pdot.h`` (ctypes; argument
marshalling only -- every step of the solver runs in libpdot.so's kernels).

The functions named ``pdot_*`` mirror the C entry points one to one and take
raw device pointers.  ``Solver`` is a convenience wrapper over them that takes
torch CUDA tensors (torch provides device memory and the stream only).

Importing this module does not load the library; the first call does, and it
raises ``PdotError`` when ``libpdot.so`` has not been built (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

F32, BF16, F64, POINTS = 0, 1, 2, 3
DIST = {"sqeuclid": 0, "l1": 1, "l2": 2, "linf": 3}
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NUMERIC, MAX_ITER, TIMEOUT, BUSY, PENDING, CANCELLED = range(10)


class PdotError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{status_str(status) if _LIB else status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int64),
        ("time_limit_s", ctypes.c_double),
        ("restart_check_every", ctypes.c_int32),
        ("adaptive_step", ctypes.c_int32),
        ("adaptive_restart", ctypes.c_int32),
        ("primal_weight_update", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("beta_suff", ctypes.c_double),
        ("beta_nec", ctypes.c_double),
        ("beta_art", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("eta0", ctypes.c_double),
        ("omega0", ctypes.c_double),
        ("R", ctypes.c_double),
        ("eps_zero", ctypes.c_double),
        ("rel_mode", ctypes.c_int32),
        ("x_dtype", ctypes.c_int32),
        ("round_plan", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("max_batch_slots", ctypes.c_int32),
        ("chunk_checks", ctypes.c_int32),
        ("batch_active_bytes", ctypes.c_uint64),
        ("pass_kernel", ctypes.c_int32),
        ("compensated_cost", ctypes.c_int32),
        ("resident", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("primal_obj", ctypes.c_double),
        ("dual_obj", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("kkt", ctypes.c_double),
        ("rel_kkt", ctypes.c_double),
        ("rel_primal", ctypes.c_double),
        ("rel_dual", ctypes.c_double),
        ("rel_gap", ctypes.c_double),
        ("iters", ctypes.c_int64),
        ("passes", ctypes.c_int64),
        ("restarts", ctypes.c_int64),
        ("rejected_steps", ctypes.c_int64),
        ("eta", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("hbm_bytes", ctypes.c_double),
        ("rounded_obj", ctypes.c_double),
        ("returned_average", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class KktParts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("rp2", "rd2", "cx", "dual", "gap", "kkt", "rel_p", "rel_d", "rel_gap", "rel_kkt")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("C", ctypes.c_void_p),
        ("c_dtype", ctypes.c_int32),
        ("ldc", ctypes.c_int64),
        ("f", ctypes.c_void_p),
        ("g", ctypes.c_void_p),
        ("tol", ctypes.c_double),
        ("X_out", ctypes.c_void_p),
        ("p_out", ctypes.c_void_p),
        ("q_out", ctypes.c_void_p),
        ("user_tag", ctypes.c_uint64),
    ]


class PointsCostDesc(ctypes.Structure):
    """pdot_points_cost: a cost generated from coordinates (c_dtype POINTS)."""
    _fields_ = [
        ("d", ctypes.c_int32),
        ("dist", ctypes.c_int32),
        ("xs", ctypes.c_void_p),
        ("ys", ctypes.c_void_p),
        ("divisor", ctypes.c_float),
    ]


class Start(ctypes.Structure):
    """pdot_start: a starting point or a saved solver state (device pointers)."""
    _fields_ = [
        ("X0", ctypes.c_void_p),
        ("p0", ctypes.c_void_p),
        ("q0", ctypes.c_void_p),
        ("state_in", ctypes.c_void_p),
        ("state_out", ctypes.c_void_p),
    ]


# Every symbol include/pdot.h declares (checked by the CPU tests).
DECLARED = [
    "pdot_default_options", "pdot_status_str", "pdot_last_error", "pdot_create", "pdot_destroy", "pdot_solve",
    "pdot_solve_host", "pdot_solve_from", "pdot_state_bytes", "pdot_resident_fits", "pdot_pdhg_steps", "pdot_kkt", "pdot_round", "pdot_dual_bound",
    "pdot_batch_submit", "pdot_poll", "pdot_cancel", "pdot_batch_pending", "pdot_launch_count", "pdot_time_pass",
    "pdot_round_noalloc", "pdot_watchdog_selftest",
]

_LIB = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libpdot.so (building it first only when asked)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise PdotError(ERR_CUDA, f"{_build.LIB} is not built; call __graft_entry__.build() or "
                                  "paper_2407_19689_gb300._build.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32
    H = ctypes.c_void_p
    sig = {
        "pdot_default_options": (None, [ctypes.POINTER(Options)]),
        "pdot_status_str": (ctypes.c_char_p, [i32]),
        "pdot_last_error": (ctypes.c_char_p, [H]),
        "pdot_create": (i32, [ctypes.POINTER(Options), i32, vp, ctypes.POINTER(H)]),
        "pdot_destroy": (i32, [H]),
        "pdot_solve": (i32, [H, i64, i64, vp, i32, i64, vp, vp, dbl, vp, vp, vp, ctypes.POINTER(Result)]),
        "pdot_solve_host": (i32, [H, i64, i64, vp, i32, i64, vp, vp, dbl, vp, vp, vp, ctypes.POINTER(Result)]),
        "pdot_solve_from": (i32, [H, i64, i64, vp, i32, i64, vp, vp, dbl, ctypes.POINTER(Start), vp, vp, vp,
                                  ctypes.POINTER(Result)]),
        "pdot_state_bytes": (i64, [i64, i64, i32]),
        "pdot_resident_fits": (i32, [i64, i64]),
        "pdot_pdhg_steps": (i32, [H, i64, i64, vp, i32, i64, vp, vp, i64, dbl, dbl, vp, vp, vp, vp, vp, vp]),
        "pdot_kkt": (i32, [H, i64, i64, vp, i32, i64, vp, vp, vp, vp, vp, ctypes.POINTER(KktParts)]),
        "pdot_round": (i32, [H, i64, i64, vp, vp, vp, vp]),
        "pdot_dual_bound": (i32, [H, i64, i64, vp, i32, i64, vp, vp, vp, vp, ctypes.POINTER(dbl)]),
        "pdot_batch_submit": (i32, [H, ctypes.POINTER(Request), i32, ctypes.POINTER(ctypes.c_uint64)]),
        "pdot_poll": (i32, [H, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result), i32,
                            ctypes.POINTER(i32)]),
        "pdot_cancel": (i32, [H, ctypes.c_uint64]),
        "pdot_batch_pending": (i32, [H, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "pdot_launch_count": (i64, [H]),
        "pdot_time_pass": (i32, [H, i64, i64, vp, i32, i64, vp, vp, i32, ctypes.POINTER(dbl),
                                 ctypes.POINTER(dbl), ctypes.POINTER(i32)]),
        "pdot_round_noalloc": (i32, [i32, vp, i64, i64, i32, vp, vp, vp, vp]),
        "pdot_watchdog_selftest": (i32, [i32, i64, ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def status_str(s: int) -> str:
    return load().pdot_status_str(int(s)).decode()


def _check(h, st: int, allow=(OK,)):
    if st not in allow:
        msg = load().pdot_last_error(h).decode() if h else ""
        raise PdotError(st, msg)
    return st


# ---------------------------------------------------------------------------
# 1:1 wrappers of the C entry points (raw pointers; ints for addresses)
# ---------------------------------------------------------------------------

def pdot_default_options() -> Options:
    o = Options()
    load().pdot_default_options(ctypes.byref(o))
    return o


def pdot_create(opts: Options | None = None, device: int = 0, stream: int = 0):
    h = ctypes.c_void_p()
    st = load().pdot_create(ctypes.byref(opts) if opts is not None else None, device, stream or None,
                            ctypes.byref(h))
    _check(None, st)
    return h


def pdot_destroy(h) -> int:
    return load().pdot_destroy(h)


def pdot_solve(h, m, n, C, c_dtype, ldc, f, g, tol, X_out=0, p_out=0, q_out=0):
    r = Result()
    st = load().pdot_solve(h, m, n, C, c_dtype, ldc, f, g, tol, X_out or None, p_out or None, q_out or None,
                           ctypes.byref(r))
    return st, r


def pdot_solve_host(h, m, n, C, c_dtype, ldc, f, g, tol, X_out=0, p_out=0, q_out=0):
    r = Result()
    st = load().pdot_solve_host(h, m, n, C, c_dtype, ldc, f, g, tol, X_out or None, p_out or None,
                                q_out or None, ctypes.byref(r))
    return st, r


def pdot_solve_from(h, m, n, C, c_dtype, ldc, f, g, tol, start: Start | None, X_out=0, p_out=0, q_out=0):
    r = Result()
    st = load().pdot_solve_from(h, m, n, C, c_dtype, ldc, f, g, tol, ctypes.byref(start) if start else None,
                                X_out or None, p_out or None, q_out or None, ctypes.byref(r))
    return st, r


def pdot_state_bytes(m, n, x_dtype) -> int:
    return load().pdot_state_bytes(m, n, x_dtype)


def pdot_resident_fits(m, n) -> int:
    return load().pdot_resident_fits(m, n)


def pdot_pdhg_steps(h, m, n, C, c_dtype, ldc, f, g, k, eta, omega, X, p, q, Xbar=0, pbar=0, qbar=0) -> int:
    return load().pdot_pdhg_steps(h, m, n, C, c_dtype, ldc, f, g, k, eta, omega, X, p, q, Xbar or None,
                                  pbar or None, qbar or None)


def pdot_kkt(h, m, n, C, c_dtype, ldc, f, g, X, p, q):
    out = KktParts()
    st = load().pdot_kkt(h, m, n, C, c_dtype, ldc, f, g, X, p, q, ctypes.byref(out))
    return st, out


def pdot_round(h, m, n, X, f, g, X_out) -> int:
    return load().pdot_round(h, m, n, X, f, g, X_out)


def pdot_dual_bound(h, m, n, C, c_dtype, ldc, f, g, p, q_out=0):
    lower = ctypes.c_double()
    st = load().pdot_dual_bound(h, m, n, C, c_dtype, ldc, f, g, p, q_out or None, ctypes.byref(lower))
    return st, lower.value


def pdot_batch_submit(h, reqs: list[Request]):
    arr = (Request * len(reqs))(*reqs)
    ids = (ctypes.c_uint64 * len(reqs))()
    st = load().pdot_batch_submit(h, arr, len(reqs), ids)
    return st, list(ids)


def pdot_poll(h, cap: int = 256):
    ids = (ctypes.c_uint64 * cap)()
    res = (Result * cap)()
    nd = ctypes.c_int32()
    st = load().pdot_poll(h, ids, res, cap, ctypes.byref(nd))
    return st, [(ids[i], res[i]) for i in range(nd.value)]


def pdot_cancel(h, ticket: int) -> int:
    return load().pdot_cancel(h, ticket)


def pdot_batch_pending(h):
    q, r = ctypes.c_int32(), ctypes.c_int32()
    st = load().pdot_batch_pending(h, ctypes.byref(q), ctypes.byref(r))
    return st, q.value, r.value


def pdot_launch_count(h) -> int:
    return load().pdot_launch_count(h)


def pdot_round_noalloc(device, stream, m, n, x_dtype, X, f, g, X_out) -> int:
    """Algorithm 3 without a handle or any allocation (scratch lives in the
    library's static device array); see include/pdot.h for the limits."""
    return load().pdot_round_noalloc(device, stream or None, m, n, x_dtype, X, f, g, X_out)


def kernel_name(variant: int, c_dtype: int) -> str:
    """Name of the pass kernel a variant code and cost type select."""
    tc = {F32: "float", BF16: "unsigned short", F64: "double", POINTS: "GenC"}.get(c_dtype, "?")
    if variant == 0:
        return f"k_pass<{tc}, ...> (register pipeline)"
    if variant == 1:
        return f"k_pass_bulk<{tc}, 8> (bulk copies per row)"
    return f"k_pass_group<{tc}, 2> (bulk copies per 4-row group)"


def pdot_watchdog_selftest(device: int = 0, polls: int = 4096):
    """Returns (status of the call, status the device reported)."""
    out = ctypes.c_int32(-1)
    st = load().pdot_watchdog_selftest(device, polls, ctypes.byref(out))
    return st, out.value


def pdot_time_pass(h, m, n, C, c_dtype, ldc, f, g, reps):
    """Returns (status, ms per pass, algorithmic bytes per pass, kernel variant)."""
    ms, b, kv = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    st = load().pdot_time_pass(h, m, n, C, c_dtype, ldc, f, g, reps, ctypes.byref(ms), ctypes.byref(b),
                               ctypes.byref(kv))
    return st, ms.value, b.value, kv.value


# ---------------------------------------------------------------------------
# torch-tensor convenience layer
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _cdtype(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported cost dtype {t.dtype}")


def _xdtype_torch(x_dtype: int):
    torch = _torch()
    return torch.float64 if x_dtype == F64 else torch.float32


class Points:
    """A cost that is never stored: C_ij = dist(xs_i, ys_j) / divisor, computed
    in FP32 by every pass from the coordinates (xs: m x d, ys: n x d, d <= 8;
    dist one of DIST).  Pass it wherever a cost matrix is accepted."""

    def __init__(self, xs, ys, dist: str = "sqeuclid", divisor: float = 1.0):
        self.xs, self.ys, self.dist, self.divisor = xs, ys, dist, float(divisor)

    @property
    def shape(self):
        return (self.xs.shape[0], self.ys.shape[0])


@dataclass
class _Cost:
    """Marshalled cost argument: pointer, dtype, leading dimension, and the
    objects that must stay alive while the library reads them."""
    ptr: int
    dtype: int
    ldc: int
    m: int
    n: int
    keep: tuple


@dataclass
class Solution:
    result: dict
    status: int
    X: object = None
    p: object = None
    q: object = None


class Solver:
    """Owns one pdot handle on a CUDA device; tensors in, tensors out."""

    def __init__(self, options: Options | None = None, device: int = 0, stream=None, **overrides):
        torch = _torch()
        self.options = options if options is not None else pdot_default_options()
        known = {name for name, _ in Options._fields_}
        for k, v in overrides.items():
            if k not in known:   # a misspelt option would otherwise be ignored silently
                raise TypeError(f"unknown solver option {k!r}")
            setattr(self.options, k, v)
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.h = pdot_create(self.options, device, stream)

    def close(self):
        if self.h is not None:
            pdot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cuda(self, t, dtype=None):
        torch = _torch()
        t = t if isinstance(t, torch.Tensor) else torch.as_tensor(t)
        if dtype is not None and t.dtype != dtype:
            t = t.to(dtype)
        return t.to(f"cuda:{self.device}").contiguous()

    def _cost(self, C) -> _Cost:
        torch = _torch()
        if isinstance(C, Points):
            xs = self._cuda(C.xs, torch.float32)
            ys = self._cuda(C.ys, torch.float32)
            if xs.dim() == 1:
                xs = xs[:, None].contiguous()
            if ys.dim() == 1:
                ys = ys[:, None].contiguous()
            if xs.dim() != 2 or ys.dim() != 2 or xs.shape[1] != ys.shape[1]:
                raise ValueError("xs and ys must be (m, d) and (n, d)")
            desc = PointsCostDesc(d=xs.shape[1], dist=DIST[C.dist], xs=xs.data_ptr(), ys=ys.data_ptr(),
                                  divisor=C.divisor)
            return _Cost(ctypes.addressof(desc), POINTS, 0, xs.shape[0], ys.shape[0], (desc, xs, ys))
        C = self._cuda(C)
        if C.dim() != 2:
            raise ValueError("C must be 2-D")
        return _Cost(C.data_ptr(), _cdtype(C), C.stride(0), C.shape[0], C.shape[1], (C,))

    def _prep(self, C, f, g):
        torch = _torch()
        c = self._cost(C)
        f = self._cuda(f, torch.float64)
        g = self._cuda(g, torch.float64)
        return c, f, g

    def state_bytes(self, m: int, n: int) -> int:
        return pdot_state_bytes(m, n, self.options.x_dtype)

    def solve(self, C, f, g, tol: float | None = None, want_plan: bool = True, X0=None, p0=None, q0=None,
              state_in=None, state_out=None) -> Solution:
        """Solve from the origin, from a starting point (X0, p0, q0; a missing
        part is 0) or from a saved state (state_in: a uint8 CUDA tensor a
        previous call filled as state_out, of state_bytes(m, n) bytes)."""
        torch = _torch()
        c, f, g = self._prep(C, f, g)
        m, n = c.m, c.n
        xt = _xdtype_torch(self.options.x_dtype)
        X = torch.empty((m, n), dtype=xt, device=f.device) if want_plan else None
        p = torch.empty(m, dtype=torch.float64, device=f.device)
        q = torch.empty(n, dtype=torch.float64, device=f.device)
        tol = tol if tol is not None else self.options.tol
        if X0 is None and p0 is None and q0 is None and state_in is None and state_out is None:
            st, r = pdot_solve(self.h, m, n, c.ptr, c.dtype, c.ldc, f.data_ptr(), g.data_ptr(), tol,
                               X.data_ptr() if X is not None else 0, p.data_ptr(), q.data_ptr())
        else:
            keep = []

            def dev(t, dtype):
                if t is None:
                    return None
                t = self._cuda(t, dtype)
                keep.append(t)
                return t.data_ptr()

            for blob in (state_in, state_out):
                if blob is not None and (not isinstance(blob, torch.Tensor) or not blob.is_cuda or
                                         blob.numel() * blob.element_size() < self.state_bytes(m, n)):
                    raise ValueError(f"state blobs must be CUDA tensors of at least {self.state_bytes(m, n)} bytes")
            start = Start(X0=dev(X0, xt), p0=dev(p0, torch.float64), q0=dev(q0, torch.float64),
                          state_in=state_in.data_ptr() if state_in is not None else None,
                          state_out=state_out.data_ptr() if state_out is not None else None)
            st, r = pdot_solve_from(self.h, m, n, c.ptr, c.dtype, c.ldc, f.data_ptr(), g.data_ptr(), tol, start,
                                    X.data_ptr() if X is not None else 0, p.data_ptr(), q.data_ptr())
        _check(self.h, st, allow=(OK, MAX_ITER, TIMEOUT, ERR_NUMERIC))
        return Solution(r.as_dict(), st, X, p, q)

    def pdhg_steps(self, C, f, g, X, p, q, k: int, eta: float, omega: float = 1.0):
        torch = _torch()
        c, f, g = self._prep(C, f, g)
        m, n = c.m, c.n
        xt = _xdtype_torch(self.options.x_dtype)
        X = self._cuda(X, xt).clone()
        p = self._cuda(p, torch.float64).clone()
        q = self._cuda(q, torch.float64).clone()
        Xb, pb, qb = torch.empty_like(X), torch.empty_like(p), torch.empty_like(q)
        st = pdot_pdhg_steps(self.h, m, n, c.ptr, c.dtype, c.ldc, f.data_ptr(), g.data_ptr(), k,
                             eta, omega, X.data_ptr(), p.data_ptr(), q.data_ptr(), Xb.data_ptr(), pb.data_ptr(),
                             qb.data_ptr())
        _check(self.h, st)
        return X, p, q, Xb, pb, qb

    def kkt(self, C, f, g, X, p, q) -> dict:
        torch = _torch()
        c, f, g = self._prep(C, f, g)
        m, n = c.m, c.n
        X = self._cuda(X, _xdtype_torch(self.options.x_dtype))
        p = self._cuda(p, torch.float64)
        q = self._cuda(q, torch.float64)
        st, out = pdot_kkt(self.h, m, n, c.ptr, c.dtype, c.ldc, f.data_ptr(), g.data_ptr(),
                           X.data_ptr(), p.data_ptr(), q.data_ptr())
        _check(self.h, st)
        return out.as_dict()

    def round(self, X, f, g):
        torch = _torch()
        X = self._cuda(X, _xdtype_torch(self.options.x_dtype))
        f = self._cuda(f, torch.float64)
        g = self._cuda(g, torch.float64)
        m, n = X.shape
        out = torch.empty_like(X)
        _check(self.h, pdot_round(self.h, m, n, X.data_ptr(), f.data_ptr(), g.data_ptr(), out.data_ptr()))
        return out

    def dual_bound(self, C, f, g, p):
        """Weak-duality lower bound f^T p + g^T q on the optimum, with
        q_j = min_i (C_ij - p_i); returns (lower, q)."""
        torch = _torch()
        c, f, g = self._prep(C, f, g)
        p = self._cuda(p, torch.float64)
        q = torch.empty(c.n, dtype=torch.float64, device=f.device)
        st, lower = pdot_dual_bound(self.h, c.m, c.n, c.ptr, c.dtype, c.ldc, f.data_ptr(), g.data_ptr(),
                                    p.data_ptr(), q.data_ptr())
        _check(self.h, st)
        return lower, q

    def launch_count(self) -> int:
        return pdot_launch_count(self.h)


class BatchSolver:
    """Continuous-batching front end over pdot_batch_submit / pdot_poll.

    ``submit`` queues one solve (torch CUDA tensors; they are kept alive until
    the ticket is reported) and returns its ticket; ``poll`` advances the
    engine by one chunk and returns the finished tickets.
    """

    def __init__(self, options: Options | None = None, device: int = 0, stream=None, **overrides):
        self.solver = Solver(options, device, stream, **overrides)
        self.h = self.solver.h
        self._keep = {}

    @property
    def options(self):
        return self.solver.options

    def close(self):
        self._keep.clear()
        self.solver.close()

    def submit(self, C, f, g, tol: float = 0.0, want_plan: bool = True, tag: int = 0) -> int:
        torch = _torch()
        c, f, g = self.solver._prep(C, f, g)
        m, n = c.m, c.n
        xt = _xdtype_torch(self.options.x_dtype)
        X = torch.empty((m, n), dtype=xt, device=f.device) if want_plan else None
        p = torch.empty(m, dtype=torch.float64, device=f.device)
        q = torch.empty(n, dtype=torch.float64, device=f.device)
        r = Request(m=m, n=n, C=c.ptr, c_dtype=c.dtype, ldc=c.ldc, f=f.data_ptr(), g=g.data_ptr(),
                    tol=tol, X_out=X.data_ptr() if X is not None else None, p_out=p.data_ptr(),
                    q_out=q.data_ptr(), user_tag=tag)
        st, ids = pdot_batch_submit(self.h, [r])
        _check(self.h, st)
        self._keep[ids[0]] = (c.keep, f, g, X, p, q)
        return ids[0]

    def poll(self, cap: int = 1024) -> list[tuple[int, Solution]]:
        st, done = pdot_poll(self.h, cap)
        _check(self.h, st)
        out = []
        for tid, r in done:
            C, f, g, X, p, q = self._keep.pop(tid, (None,) * 6)
            out.append((tid, Solution(r.as_dict(), r.status, X, p, q)))
        return out

    def cancel(self, ticket: int) -> int:
        return pdot_cancel(self.h, ticket)

    def pending(self) -> tuple[int, int]:
        st, q, r = pdot_batch_pending(self.h)
        return q, r

    def run(self) -> dict:
        """Poll until every submitted ticket is reported."""
        res = {}
        while True:
            for tid, sol in self.poll():
                res[tid] = sol
            q, r = self.pending()
            if q == 0 and r == 0:
                for tid, sol in self.poll():
                    res[tid] = sol
                return res
