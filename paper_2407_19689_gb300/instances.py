"""Seeded synthetic OT instances (inputs only; no solver arithmetic lives here).

Both the CUDA path and the FP64 oracle take their inputs from this module, so
it imports nothing from either.  Every draw comes from numpy's PCG64 generator
(``np.random.default_rng(seed)``) in FP64 before any cast.

Workloads (the paper's DOTmark images are not available; these stand in for
them with the paper's shapes, Table 2, and its grid-coordinate costs, Sec. 5.1):

- ``points_instance``: m source and n target points i.i.d. uniform in [0,1]^d,
  cost squared Euclidean or L1, marginals uniform(0.1, 1) or Dirichlet(alpha),
  normalised to sum 1.
- ``grid_blob_instance``: a G x G pixel grid on both sides (m = n = G^2),
  marginals = mixtures of 3-8 Gaussian blobs (sigma 2-10 px, weights
  U(0.5, 1.5)) plus a 1e-4 floor, normalised; cost = squared grid distance
  scaled to [0, 1] (or the paper's l1 / l2 / l_inf pixel distances).
- ``batch_sizes`` / ``serve_requests``: the size/arrival mixes of the batched
  and served workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20240727


def seed_for(config_index: int, instance_index: int = 0) -> int:
    return SEED_BASE + 1000 * config_index + instance_index


def _normalise(w: np.ndarray) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    return w / w.sum()


def cost_from_points(xs: np.ndarray, ys: np.ndarray, kind: str = "sqeuclid") -> np.ndarray:
    """Cost matrix between two point clouds (rows = xs, columns = ys), FP64."""
    diff = xs[:, None, :] - ys[None, :, :]
    if kind == "sqeuclid":
        return np.einsum("ijk,ijk->ij", diff, diff)
    if kind == "l1":
        return np.abs(diff).sum(axis=2)
    if kind == "l2":
        return np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    if kind == "linf":
        return np.abs(diff).max(axis=2)
    raise ValueError(kind)


@dataclass
class Instance:
    C: np.ndarray     # (m, n) float64
    f: np.ndarray     # (m,) float64, sums to 1
    g: np.ndarray     # (n,) float64, sums to 1
    name: str = ""


def points_instance(m: int, n: int, seed: int, d: int = 2, cost: str = "sqeuclid",
                    marginals: str = "uniform", alpha: float = 1.0, scale_to_unit: bool = False) -> Instance:
    rng = np.random.default_rng(seed)
    xs = rng.random((m, d))
    ys = rng.random((n, d))
    if marginals == "uniform":
        f = _normalise(rng.uniform(0.1, 1.0, m))
        g = _normalise(rng.uniform(0.1, 1.0, n))
    elif marginals == "dirichlet":
        f = _normalise(rng.dirichlet(np.full(m, alpha)))
        g = _normalise(rng.dirichlet(np.full(n, alpha)))
    elif marginals == "equal":
        f = np.full(m, 1.0 / m)
        g = np.full(n, 1.0 / n)
    else:
        raise ValueError(marginals)
    C = cost_from_points(xs, ys, cost)
    if scale_to_unit:
        C = C / C.max()
    return Instance(C, f, g, f"points_{m}x{n}_{cost}")


def blob_marginal(G: int, rng: np.random.Generator) -> np.ndarray:
    K = int(rng.integers(3, 9))
    a, b = np.meshgrid(np.arange(G, dtype=np.float64), np.arange(G, dtype=np.float64), indexing="ij")
    dens = np.zeros((G, G))
    for _ in range(K):
        ca, cb = rng.uniform(0, G - 1, 2)
        s = rng.uniform(2.0, 10.0)
        w = rng.uniform(0.5, 1.5)
        dens += w * np.exp(-((a - ca) ** 2 + (b - cb) ** 2) / (2.0 * s * s))
    dens /= dens.max()
    dens += 1e-4
    return _normalise(dens.reshape(-1))


def grid_coords(G: int) -> np.ndarray:
    a, b = np.meshgrid(np.arange(G, dtype=np.float64), np.arange(G, dtype=np.float64), indexing="ij")
    return np.stack([a.reshape(-1), b.reshape(-1)], axis=1)


def grid_cost(G: int, kind: str = "sqeuclid", scale_to_unit: bool = True) -> np.ndarray:
    P = grid_coords(G)
    C = cost_from_points(P, P, kind)
    if scale_to_unit:
        C = C / C.max()
    return C


def grid_blob_instance(G: int, seed: int, cost: str = "sqeuclid", build_cost: bool = True) -> Instance:
    rng = np.random.default_rng(seed)
    f = blob_marginal(G, rng)
    g = blob_marginal(G, rng)
    C = grid_cost(G, cost) if build_cost else None
    return Instance(C, f, g, f"grid{G}_{cost}")


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 2048) -> list[tuple[int, int]]:
    """m, n drawn independently log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append((m, n))
    return out


def batch_instance(m: int, n: int, seed: int) -> Instance:
    """Batched workload: U[0,1]^2 points, squared-Euclidean cost, Dirichlet(1) marginals."""
    return points_instance(m, n, seed, d=2, cost="sqeuclid", marginals="dirichlet", alpha=1.0)


@dataclass
class Request:
    arrival_s: float
    m: int
    n: int
    d: int
    cost: str
    alpha: float
    tol: float
    seed: int


def serve_requests(count: int, rate_per_s: float, seed: int, lo: int = 128, hi: int = 8192) -> list[Request]:
    """Poisson arrivals; sizes log-uniform in [lo, hi]; d in {2,3,8}; cost sq-Euclidean or L1
    (50/50, scaled to [0,1] by its max); Dirichlet(alpha), alpha ~ U(0.5, 2); tol 1e-4 or 1e-6."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        m = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        d = int(rng.choice([2, 3, 8]))
        cost = "sqeuclid" if rng.random() < 0.5 else "l1"
        alpha = float(rng.uniform(0.5, 2.0))
        tol = 1e-4 if rng.random() < 0.5 else 1e-6
        out.append(Request(t, m, n, d, cost, alpha, tol, seed * 7919 + k))
    return out


def request_instance(r: Request) -> Instance:
    return points_instance(r.m, r.n, r.seed, d=r.d, cost=r.cost, marginals="dirichlet",
                           alpha=r.alpha, scale_to_unit=True)


def device_cost_from_points(xs, ys, kind: str = "sqeuclid", scale_to_unit: bool = False, dtype=None):
    """Cost matrix between two point clouds built on the GPU with torch ops
    (input generation for the served workload; FP64, cast at the end)."""
    import torch
    x = torch.as_tensor(xs, dtype=torch.float64)
    y = torch.as_tensor(ys, dtype=torch.float64)
    if kind == "sqeuclid":
        C = torch.cdist(x, y, p=2.0) ** 2
    elif kind == "l1":
        C = torch.cdist(x, y, p=1.0)
    else:
        raise ValueError(kind)
    if scale_to_unit:
        C = C / C.max()
    return C.to(dtype) if dtype is not None else C


def request_points(r: "Request"):
    """Points and marginals of a served request (same draws as request_instance)."""
    rng = np.random.default_rng(r.seed)
    xs = rng.random((r.m, r.d))
    ys = rng.random((r.n, r.d))
    f = _normalise(rng.dirichlet(np.full(r.m, r.alpha)))
    g = _normalise(rng.dirichlet(np.full(r.n, r.alpha)))
    return xs, ys, f, g
