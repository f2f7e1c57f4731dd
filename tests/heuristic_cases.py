"""Hand-derived and pinned-step special cases of the Sec. 5 heuristics,
shared by the oracle's pins (tests/test_oracle_pins.py) and their GPU twins
(tests/test_gpu_parity.py).  Every expected value here is derived from the
rule's statement on a tiny instance, or composed from the oracle's pinned
building blocks (one Algorithm 2 step, the KKT error); none comes from the
CUDA path.
"""
import math

import numpy as np

from paper_2407_19689_gb300 import instances as I


def step_rule_from_origin_case():
    """1 x 1, C = 1, f = g = 1 from the origin (reading C1) with eta0 = 1.
    Pass 1: X stays 0 (dX = 0, eta_bar = inf): accepted, p = q = 1,
    eta1 = 1 + 2^-0.6.  Pass 2 (t = 3): the reduced cost is 1 - 2 = -1, so
    X+ = eta1 =: d and (2X+ - X) 1 = 2d; p+ = q+ = 1 + eta1 (1 - 2d).
    dX = d, dp = dq = eta1 (1 - 2d), hence
    eta_bar = (d^2 + 2 eta1^2 (1 - 2d)^2) / (4 |eta1 (1 - 2d) d|)
            = (1 + 2 (1 - 2d)^2) / (4 |1 - 2d|)      (d = eta1)
            = 1.2675... < eta1 = 1.6598...: rejected, and
    eta2 = min((1 - 3^-0.3) eta_bar, (1 + 3^-0.6) eta1).
    Returns (data, expected final eta); shared with the GPU twin."""
    eta1 = 1 + 2 ** -0.6
    d = eta1
    eta_bar = (1 + 2 * (1 - 2 * d) ** 2) / (4 * abs(1 - 2 * d))
    assert eta_bar < eta1
    return ([[1.0]], [1.0], [1.0]), min((1 - 3 ** -0.3) * eta_bar, (1 + 3 ** -0.6) * eta1)


def check_candidates(ora, ins, K, eta, nchecks, start=None):
    """Constant-step Algorithm 2 from `start` (the origin by default) without
    restarts, from pinned steps and the pinned KKT error: at every K-th step,
    the restart candidate (the current iterate if its KKT error is strictly
    smaller than the uniform average's, else the average; reading C13) and
    that KKT error.  Returns (KKT of the start, [(candidate, KKT), ...])."""
    m, n = ins.C.shape
    X, p, q = start if start is not None else (np.zeros((m, n)), np.zeros(m), np.zeros(n))
    k0 = ora.kkt(ins.C, ins.f, ins.g, X, p, q).kkt
    its, out = [], []
    for _ in range(nchecks):
        for _ in range(K):
            X, p, q = ora.pdhg_step(ins.C, ins.f, ins.g, X, p, q, eta, eta)
            its.append((X, p, q))
        avg = tuple(np.mean([z[i] for z in its], axis=0) for i in range(3))
        kc = ora.kkt(ins.C, ins.f, ins.g, X, p, q).kkt
        ka = ora.kkt(ins.C, ins.f, ins.g, *avg).kkt
        out.append(((X, p, q), kc) if kc < ka else (avg, ka))
    return k0, out


RESTART_PIN = dict(seed=161, m=9, n=7, K=8, eta=0.1)


def restart_condition_case(ora, which):
    """Options of the condition-(i)-alone or condition-(ii)-alone run, the
    1-based check j at which the condition first holds, and the candidate the
    solve must return when its pass budget ends one check after that restart
    (the next K steps from the restart point, fresh average).

    (i): KKT(candidate) <= beta_suff KKT(restart point).  beta_suff is put
    geometrically halfway between the ratio at check 3 and the smallest ratio
    before it, so (i) first holds at check 3.
    (ii): KKT(candidate) <= beta_nec KKT(restart point) and KKT(candidate) >
    KKT(candidate of the previous check) (reading C8; the restart point's KKT
    at the first check).  With beta_nec = 0.9 it first holds where the
    candidates' KKT error first rises."""
    ins = I.points_instance(RESTART_PIN["m"], RESTART_PIN["n"], RESTART_PIN["seed"])
    K, eta = RESTART_PIN["K"], RESTART_PIN["eta"]
    k0, seq = check_candidates(ora, ins, K, eta, 6)
    kk = [c[1] for c in seq]
    base = dict(tol=0.0, check_every=K, adaptive_step=0, adaptive_restart=1, primal_weight_update=0, eta0=eta,
                beta_art=1e9)
    if which == "i":
        j = 3
        assert kk[j - 1] < 0.9 * min(kk[: j - 1])
        beta = math.sqrt(kk[j - 1] * min(kk[: j - 1])) / k0
        opts = dict(base, beta_suff=beta, beta_nec=0.0)
    else:
        prev = [k0] + kk[:-1]
        rises = [i for i in range(6) if kk[i] > prev[i] and kk[i] <= 0.9 * k0]
        j = rises[0] + 1
        assert kk[j - 1] > 1.01 * prev[j - 1]            # a clear rise, not a tie
        assert all(kk[i] < 0.99 * prev[i] for i in range(j - 1))
        opts = dict(base, beta_suff=0.0, beta_nec=0.9)
    _, after = check_candidates(ora, ins, K, eta, 1, start=seq[j - 1][0])
    return ins, opts, j, after[0][0]


# One-pass cases of the step-size rule (reading C6), derived by hand.  With
# m = n = 1 (or m = 2, n = 1) one Algorithm 2 step is a handful of scalar
# operations, so eta_bar, the accept/reject decision and the next step size
# follow from the rule's statement:
#   eta_bar = (omega ||dX||^2 + ||(dp, dq)||^2 / omega) / (2 |dp^T dX 1 + dq^T dX^T 1|),
#   accept iff eta <= eta_bar,  eta' = min((1 - t^-0.3) eta_bar, (1 + t^-0.6) eta),
# t = 2 + (iterations accepted so far); eta' is used next either way.  Each
# case: data, starting point, (eta0, omega0), and the expected (iters,
# rejected), final eta and final point after one pass.
STEP_RULE_CASES = [
    # "reject": C = 1, f = g = 1, start X = 5/2, p = q = 0, eta = omega = 1.
    # X+ = 5/2 - (1 - 0 - 0) = 3/2; (2X+ - X) 1 = 1/2, so p+ = q+ = 1 - 1/2 = 1/2.
    # dX = -1, dp = dq = 1/2: ||dX||^2 = 1, ||dy||^2 = 1/2, dy^T A dx = -1,
    # eta_bar = (1 + 1/2) / 2 = 3/4 < eta: rejected, the state is kept,
    # eta' = min((1 - 2^-0.3) 3/4, (1 + 2^-0.6) 1) = (1 - 2^-0.3) 3/4.
    dict(name="reject", C=[[1.0]], f=[1.0], g=[1.0], X0=[[2.5]], p0=[0.0], q0=[0.0], eta0=1.0, omega0=1.0,
         iters=0, rejected=1, eta=0.75 * (1 - 2 ** -0.3), X=[[2.5]], p=[0.0], q=[0.0]),
    # "accept, omega = 2": same data, start X = 5/2, p = q = 0, eta = 1/2 (tau = 1/4, sigma = 1).
    # X+ = 5/2 - 1/4 = 9/4; (2X+ - X) 1 = 2, so p+ = q+ = 1 - 2 = -1.
    # dX = -1/4, dp = dq = -1: omega ||dX||^2 = 1/8, ||dy||^2 / omega = 1, dy^T A dx = 1/2,
    # eta_bar = (1/8 + 1) / 1 = 9/8 >= eta: accepted, eta' = min((1 - 2^-0.3) 9/8, (1 + 2^-0.6) / 2)
    # = (1 - 2^-0.3) 9/8.  (omega on the other two terms would give eta_bar = 4 + 1/32.)
    dict(name="accept_omega2", C=[[1.0]], f=[1.0], g=[1.0], X0=[[2.5]], p0=[0.0], q0=[0.0], eta0=0.5, omega0=2.0,
         iters=1, rejected=0, eta=1.125 * (1 - 2 ** -0.3), X=[[2.25]], p=[-1.0], q=[-1.0]),
    # "two sources": m = 2, n = 1, C = [1; 0], f = [1/2; 1/2], g = 1, start X = [1; 1], p = q = 0,
    # eta = omega = 1.  X+ = [max(0, 1 - 1); max(0, 1 - 0)] = [0; 1]; 2X+ - X = [-1; 1] has row sums
    # [-1; 1] and column sum 0, so p+ = [3/2; -1/2], q+ = 1.  dX = [-1; 0], dp = [3/2; -1/2], dq = 1:
    # ||dX||^2 = 1, ||dy||^2 = 9/4 + 1/4 + 1 = 7/2, dy^T A dx = (3/2)(-1) + (-1/2)(0) + (1)(-1) = -5/2,
    # eta_bar = (1 + 7/2) / 5 = 9/10 < eta: rejected, eta' = (1 - 2^-0.3) 9/10.
    # (Without the column part dq^T dX^T 1, eta_bar would be 3/2: accepted.)
    dict(name="two_sources", C=[[1.0], [0.0]], f=[0.5, 0.5], g=[1.0], X0=[[1.0], [1.0]], p0=[0.0, 0.0], q0=[0.0],
         eta0=1.0, omega0=1.0, iters=0, rejected=1, eta=0.9 * (1 - 2 ** -0.3), X=[[1.0], [1.0]], p=[0.0, 0.0],
         q=[0.0]),
]
