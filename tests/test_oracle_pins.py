"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test names the passage it pins.  None of them retypes the oracle's own
formula: they use closed forms (Prop. 1, 1-D W1, separable costs), brute force
(Birkhoff), library solvers (scipy's assignment and HiGHS LP), the explicit
Kronecker matrix of Eq. (4) with the generic Algorithm 1, and invariants
(fixed point at an optimum, scaling by the data precision, Lemma 2).
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2407_19689_gb300 import instances as I
from heuristic_cases import STEP_RULE_CASES, restart_condition_case, step_rule_from_origin_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ot_closed_forms.txt")


def _rand_instance(m, n, seed, marg="uniform"):
    return I.points_instance(m, n, seed, marginals=marg)


# --------------------------------------------------------------------------
# Eq. (4) and Prop. 1: the implicit operator pair
# --------------------------------------------------------------------------

def _kron_A(m, n):
    """A = [1_n^T (x) I_m ; I_n (x) 1_m^T] of Eq. (4) (vec stacks columns)."""
    return np.vstack([np.kron(np.ones((1, n)), np.eye(m)), np.kron(np.eye(n), np.ones((1, m)))])


def test_operators_match_kronecker_matrix(ora):
    """Eq. (4): A vec(X) = [X1; X^T1] and A^T[p;q] = p1^T + 1q^T, against np.kron."""
    rng = np.random.default_rng(1)
    m, n = 5, 7
    A = _kron_A(m, n)
    X = rng.standard_normal((m, n))
    p, q = rng.standard_normal(m), rng.standard_normal(n)
    r, c = ora.apply_A(X)
    ax = A @ X.reshape(-1, order="F")
    np.testing.assert_allclose(np.concatenate([r, c]), ax, rtol=0, atol=1e-13)
    aty = A.T @ np.concatenate([p, q])
    np.testing.assert_allclose(ora.apply_At(p, q).reshape(-1, order="F"), aty, rtol=0, atol=1e-13)


def test_operator_adjointness(ora):
    rng = np.random.default_rng(2)
    m, n = 33, 17
    X = rng.standard_normal((m, n))
    p, q = rng.standard_normal(m), rng.standard_normal(n)
    r, c = ora.apply_A(X)
    lhs = r @ p + c @ q
    rhs = np.sum(X * ora.apply_At(p, q))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("m,n", [(3, 4), (16, 9), (40, 40)])
def test_operator_norm_is_sqrt_m_plus_n(ora, m, n):
    """Prop. 1: ||A||_2 = sqrt(m+n), attained at X = 1/sqrt(mn)."""
    rng = np.random.default_rng(3)
    X = rng.random((m, n))
    for _ in range(200):
        r, c = ora.apply_A(X)
        X = ora.apply_At(r, c)
        X /= np.linalg.norm(X)
    r, c = ora.apply_A(X)
    est = math.sqrt(r @ r + c @ c)
    assert abs(est - math.sqrt(m + n)) < 1e-9
    U = np.full((m, n), 1.0 / math.sqrt(m * n))
    r, c = ora.apply_A(U)
    assert abs(math.sqrt(r @ r + c @ c) - math.sqrt(m + n)) < 1e-12


# --------------------------------------------------------------------------
# Algorithm 2 step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(2, 3), (4, 4), (6, 5)])
def test_alg2_step_equals_alg1_with_explicit_A(ora, m, n):
    """Sec. 3 (vectorisation): Algorithm 2's iterates equal Algorithm 1's on
    c = vec(C), b = [f; g] and the explicit Kronecker A."""
    ins = _rand_instance(m, n, 10 + m)
    rng = np.random.default_rng(4)
    X = rng.random((m, n)) * 0.1
    p, q = rng.standard_normal(m) * 0.1, rng.standard_normal(n) * 0.1
    # tau != sigma (a primal weight omega = 0.6), so a swapped step size fails here
    tau, sigma = 0.3 / math.sqrt(m + n), 0.5 / math.sqrt(m + n)
    A = _kron_A(m, n)
    for _ in range(5):
        Xn, pn, qn = ora.pdhg_step(ins.C, ins.f, ins.g, X, p, q, tau, sigma)
        xn, yn = ora.lp_pdhg_step(A, np.concatenate([ins.f, ins.g]), ins.C.reshape(-1, order="F"),
                                  X.reshape(-1, order="F"), np.concatenate([p, q]), tau, sigma)
        np.testing.assert_allclose(Xn.reshape(-1, order="F"), xn, rtol=0, atol=1e-14)
        np.testing.assert_allclose(np.concatenate([pn, qn]), yn, rtol=0, atol=1e-14)
        X, p, q = Xn, pn, qn


def test_optimum_is_fixed_point_of_step(ora):
    """An optimal (X*, p*, q*) solves the minimax, so one PDHG step leaves it in place."""
    ins = _rand_instance(9, 11, 21)
    obj, X, p, q = ora.exact_transport(ins.C, ins.f, ins.g)
    for tau, sigma in [(0.1, 0.1), (0.01, 3.0)]:
        Xn, pn, qn = ora.pdhg_step(ins.C, ins.f, ins.g, X, p, q, tau, sigma)
        np.testing.assert_allclose(Xn, X, rtol=0, atol=1e-15)
        np.testing.assert_allclose(pn, p, rtol=0, atol=1e-13)
        np.testing.assert_allclose(qn, q, rtol=0, atol=1e-13)


def test_scaling_by_data_precision_is_exact(ora):
    """Sec. 4.2: iterates on (C, f, g)/Delta are the iterates on (C, f, g) divided by
    Delta at the same steps; with Delta a power of two this holds bit for bit."""
    ins = _rand_instance(7, 6, 31)
    z0 = (np.zeros((7, 6)), np.zeros(7), np.zeros(6))
    a = ora.pdhg_steps(ins.C, ins.f, ins.g, *z0, k=25, eta=0.2)
    s = 2.0 ** -7
    b = ora.pdhg_steps(ins.C * s, ins.f * s, ins.g * s, *z0, k=25, eta=0.2)
    for u, v in zip(a, b):
        assert np.array_equal(u * s, v)
    # The whole adaptive solve (restarts, steps, primal weight) is scale-equivariant
    # too, once the two absolute constants scale with the data: R (a bound on
    # ||z||; <C,X> - f^T p - g^T q is quadratic in the scaling, so gap/R stays
    # linear) and eps_zero of the primal-weight update.  Every decision then
    # compares ratios of homogeneous quantities.
    ra = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=0.0, max_passes=640, R=1.0, eps_zero=1e-10))
    rb = ora.solve(ins.C * s, ins.f * s, ins.g * s, ora.Options(tol=0.0, max_passes=640, R=s, eps_zero=1e-10 * s))
    assert ra.restarts >= 3
    assert (ra.restarts, ra.rejected, ra.iters) == (rb.restarts, rb.rejected, rb.iters)
    assert np.array_equal(ra.X * s, rb.X) and np.array_equal(ra.p * s, rb.p)


# --------------------------------------------------------------------------
# KKT error (Sec. 3.1)
# --------------------------------------------------------------------------

def test_kkt_closed_forms(ora):
    ins = _rand_instance(8, 5, 41)
    C, f, g = ins.C, ins.f, ins.g
    # At the origin only the primal residual is left (C >= 0 so [-C]^+ = 0).
    k0 = ora.kkt(C, f, g, np.zeros((8, 5)), np.zeros(8), np.zeros(5))
    assert abs(k0.kkt - math.sqrt(np.sum(f ** 2) + np.sum(g ** 2))) < 1e-15
    # The product plan f g^T is feasible; with zero duals only the gap <C, f g^T> is left.
    kp = ora.kkt(C, f, g, np.outer(f, g), np.zeros(8), np.zeros(5), R=2.0)
    assert abs(kp.kkt - abs(f @ C @ g) / 2.0) < 1e-14
    # Constant duals p = t 1: dual infeasibility sum_ij ([t - C_ij]^+)^2.
    t = 0.4
    kd = ora.kkt(C, f, g, np.outer(f, g), np.full(8, t), np.zeros(5))
    assert abs(kd.rd2 - np.sum(np.maximum(t - C, 0.0) ** 2)) < 1e-14
    assert abs(kd.dual - t) < 1e-15
    # At an exact optimum every part vanishes.
    obj, X, p, q = ora.exact_transport(C, f, g)
    ks = ora.kkt(C, f, g, X, p, q)
    assert ks.kkt < 1e-14 and ks.rel_kkt < 1e-13


def test_relative_measures_closed_forms(ora):
    """Reading C5 at points where each relative part reduces to a constant:
    at the origin the primal residual is [f; g] itself (rel_p = 1, or
    |b| / (1 + |b|) with the '1 +' denominators) and the duals are feasible
    with a zero gap; at the product plan f g^T with zero duals the plan is
    feasible and the whole objective is gap (rel_gap = 1, or <C,X> / (1 + <C,X>))."""
    ins = _rand_instance(8, 5, 42)
    C, f, g = ins.C, ins.f, ins.g
    nb = math.sqrt(np.sum(f ** 2) + np.sum(g ** 2))
    z = (np.zeros((8, 5)), np.zeros(8), np.zeros(5))
    k0, k1 = ora.kkt(C, f, g, *z), ora.kkt(C, f, g, *z, rel_mode=1)
    assert abs(k0.rel_p - 1.0) < 1e-15 and k0.rel_d == 0.0 and k0.rel_gap == 0.0 and k0.rel_kkt == k0.rel_p
    assert abs(k1.rel_p - nb / (1.0 + nb)) < 1e-15 and k1.rel_d == 0.0 and k1.rel_gap == 0.0
    P = np.outer(f, g)
    cx = f @ C @ g
    k0, k1 = ora.kkt(C, f, g, P, z[1], z[2]), ora.kkt(C, f, g, P, z[1], z[2], rel_mode=1)
    assert k0.rel_p < 1e-15 and k0.rel_d == 0.0 and abs(k0.rel_gap - 1.0) < 1e-15
    assert abs(k1.rel_gap - cx / (1.0 + cx)) < 1e-15 and abs(k0.rel_kkt - 1.0) < 1e-15
    # X = 0 with a feasible dual p = t 1 (t <= min C): the whole dual objective t
    # is gap and nothing else contributes to it (rel_gap = 1, or t / (1 + t)).
    t = 0.5 * C.min()
    assert t > 0.0
    k0, k1 = ora.kkt(C, f, g, z[0], np.full(8, t), z[2]), ora.kkt(C, f, g, z[0], np.full(8, t), z[2], rel_mode=1)
    assert k0.rd2 == 0.0 and abs(k0.rel_gap - 1.0) < 1e-15 and abs(k1.rel_gap - t / (1.0 + t)) < 1e-15


def test_gap_is_weak_duality_slack(ora):
    """Eq. (1) and its dual: for a feasible plan X (X1 = f, X^T1 = g) and a
    feasible dual (p_i + q_j <= C_ij) the gap <C,X> - f^T p - g^T q equals
    sum_ij X_ij (C_ij - p_i - q_j) >= 0 (weak duality; it vanishes exactly
    under complementary slackness)."""
    ins = _rand_instance(8, 5, 46)
    C, f, g = ins.C, ins.f, ins.g
    X = 0.5 * ora.exact_transport(C, f, g)[1] + 0.5 * np.outer(f, g)
    p = np.random.default_rng(47).standard_normal(8) * 0.1
    q = (C - p[:, None]).min(axis=0)
    k = ora.kkt(C, f, g, X, p, q)
    slack = np.sum(X * (C - p[:, None] - q[None, :]))
    assert k.rd2 < 1e-30 and slack > 0.0
    assert abs(k.gap - slack) < 1e-14


def test_relative_measures_scale_with_their_own_data(ora):
    """Reading C5: each relative part is measured against the data it refers
    to -- the primal part against the marginals only, the dual part against the
    cost only: rel_p does not move when C changes, rel_d does not move when
    the marginals change, and doubling C (marginals) halves rel_d (rel_p)
    when the residual itself is unchanged."""
    ins, other = _rand_instance(8, 5, 43), _rand_instance(8, 5, 44)
    rng = np.random.default_rng(45)
    X = rng.random((8, 5)) * 0.05
    p, q = rng.standard_normal(8) * 0.3, rng.standard_normal(5) * 0.3
    for mode in (0, 1):
        a = ora.kkt(ins.C, ins.f, ins.g, X, p, q, rel_mode=mode)
        b = ora.kkt(other.C, ins.f, ins.g, X, p, q, rel_mode=mode)
        c = ora.kkt(ins.C, other.f, other.g, X, p, q, rel_mode=mode)
        assert a.rel_d > 0.0 and a.rel_p > 0.0
        assert b.rel_p == a.rel_p and c.rel_d == a.rel_d
    # C -> 2C with p, q -> 2p, 2q doubles the dual residual and ||C||_F alike.
    a = ora.kkt(ins.C, ins.f, ins.g, X, p, q)
    d = ora.kkt(2.0 * ins.C, ins.f, ins.g, X, 2.0 * p, 2.0 * q)
    assert d.rel_d == a.rel_d and d.rd2 == 4.0 * a.rd2


# --------------------------------------------------------------------------
# Exact optimum of Eq. (1)
# --------------------------------------------------------------------------

def _golden():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, mn, C, f, g, opt = [s.strip() for s in line.split("|")]
        m, n = map(int, mn.split())
        out.append((name, np.array(C.split(), float).reshape(m, n), np.array(f.split(), float),
                    np.array(g.split(), float), float(opt)))
    return out


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c[0])
def test_exact_transport_golden(ora, case):
    name, C, f, g, opt = case
    obj, X, p, q = ora.exact_transport(C, f, g)
    assert abs(obj - opt) < 1e-14
    res = ora.solve(C, f, g, ora.Options(tol=1e-10))
    assert res.status == 0 and abs(res.primal_obj - opt) < 1e-8


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_exact_transport_vs_brute_force(ora, n):
    """Birkhoff: with f = g = 1/n the optimum is a permutation / n."""
    ins = I.points_instance(n, n, 50 + n, marginals="equal")
    best = min(sum(ins.C[i, s[i]] for i in range(n)) for s in itertools.permutations(range(n))) / n
    obj, *_ = ora.exact_transport(ins.C, ins.f, ins.g)
    assert abs(obj - best) < 1e-14


def test_exact_transport_vs_hungarian(ora):
    sp = pytest.importorskip("scipy.optimize")
    n = 60
    ins = I.points_instance(n, n, 61, marginals="equal")
    ri, ci = sp.linear_sum_assignment(ins.C)
    obj, *_ = ora.exact_transport(ins.C, ins.f, ins.g)
    assert abs(obj - ins.C[ri, ci].sum() / n) < 1e-13


@pytest.mark.parametrize("m,n,seed", [(9, 13, 71), (20, 7, 72), (25, 25, 73)])
def test_exact_transport_vs_highs(ora, m, n, seed):
    sp = pytest.importorskip("scipy.optimize")
    ins = I.points_instance(m, n, seed, marginals="dirichlet", alpha=1.0)
    A = _kron_A(m, n)
    lp = sp.linprog(ins.C.reshape(-1, order="F"), A_eq=A, b_eq=np.concatenate([ins.f, ins.g]),
                    bounds=(0, None), method="highs")
    obj, *_ = ora.exact_transport(ins.C, ins.f, ins.g)
    assert abs(obj - lp.fun) < 1e-9


def test_exact_transport_one_dimensional_w1(ora):
    """1-D closed form: with cost |x - y|, OPT = integral |F(t) - G(t)| dt."""
    rng = np.random.default_rng(81)
    x, y = rng.random(23), rng.random(31)
    f, g = rng.dirichlet(np.ones(23)), rng.dirichlet(np.ones(31))
    C = np.abs(x[:, None] - y[None, :])
    pts = np.sort(np.concatenate([x, y]))
    F = np.array([f[x <= t].sum() for t in pts[:-1]])
    G = np.array([g[y <= t].sum() for t in pts[:-1]])
    w1 = np.sum(np.abs(F - G) * np.diff(pts))
    obj, *_ = ora.exact_transport(C, f, g)
    assert abs(obj - w1) < 1e-13


def test_exact_transport_certificates(ora):
    """Primal feasibility, dual feasibility, zero gap, complementary slackness."""
    ins = I.points_instance(40, 30, 91, marginals="dirichlet", alpha=0.5)
    obj, X, p, q = ora.exact_transport(ins.C, ins.f, ins.g)
    assert X.min() >= 0.0
    np.testing.assert_allclose(X.sum(1), ins.f, atol=1e-15)
    np.testing.assert_allclose(X.sum(0), ins.g, atol=1e-15)
    red = ins.C - p[:, None] - q[None, :]
    assert red.min() > -1e-14
    assert abs(obj - (ins.f @ p + ins.g @ q)) < 1e-14
    assert np.all(np.abs(red[X > 0]) < 1e-14)


# --------------------------------------------------------------------------
# The solve (Algorithm 2 + Sec. 5)
# --------------------------------------------------------------------------

def _certified_interval(C, f, g, X, p, q):
    """OPT lies in [dual bound, primal bound]: a feasible dual by lowering q
    (q_j <- min_i C_ij - p_i) and a feasible plan by Algorithm 3 (Lemma 2)."""
    qf = np.minimum(q, (C - p[:, None]).min(axis=0))
    return f @ p + g @ qf


@pytest.mark.parametrize("m,n,seed", [(64, 64, I.seed_for(0)), (37, 51, 101), (80, 20, 102)])
def test_solve_reaches_exact_optimum(ora, m, n, seed):
    ins = I.points_instance(m, n, seed)
    opt, *_ = ora.exact_transport(ins.C, ins.f, ins.g)
    for tol, bound in [(1e-4, 5e-3), (1e-6, 1e-5), (1e-8, 1e-7)]:
        res = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=tol))
        assert res.status == 0 and res.rel_kkt <= tol
        # the measures the solve reports are those of the iterate it returns
        k = ora.kkt(ins.C, ins.f, ins.g, res.X, res.p, res.q)
        for part in ("rel_p", "rel_d", "rel_gap", "rel_kkt"):
            assert abs(getattr(res, part) - getattr(k, part)) <= 1e-12 * getattr(k, part) + 1e-300, part
        assert abs(res.primal_obj - opt) / opt < bound
        lb = _certified_interval(ins.C, ins.f, ins.g, res.X, res.p, res.q)
        ub = ins.C.reshape(-1) @ ora.round_plan(res.X, ins.f, ins.g).reshape(-1)
        assert lb <= opt + 1e-15 and opt <= ub + 1e-15


def test_solve_theory_mode_identifies_support(ora):
    """Constant eta = 1/(2 sqrt(m+n)), fixed-beta restarts to the average
    (Eq. 6): converges; after identification X_ij is exactly 0 on N (Thm. 1)."""
    ins = I.points_instance(12, 10, 111)
    opt, Xs, ps, qs = ora.exact_transport(ins.C, ins.f, ins.g)
    opts = ora.Options(tol=1e-9, adaptive_step=0, adaptive_restart=0, primal_weight_update=0, beta=0.2,
                       max_passes=2_000_000)
    res = ora.solve(ins.C, ins.f, ins.g, opts)
    assert res.status == 0
    assert abs(res.primal_obj - opt) / opt < 1e-7
    # the constant step is Theorem 1's 1 / (2 ||A||_2), ||A||_2 = sqrt(m + n) (Prop. 1)
    assert abs(res.eta - 0.5 / math.sqrt(12 + 10)) < 1e-16
    N = (ins.C - ps[:, None] - qs[None, :]) > 1e-6
    assert np.all(res.X[N] == 0.0)


def test_solve_average_is_the_uniform_mean_of_the_iterates(ora):
    """Algorithm 2's running average (reading C7: uniform weights): with a
    constant step and no restart (fixed-beta test with beta = 0 never fires),
    the candidate the solve returns at its pass limit is the average, which
    must equal the plain mean of the iterates of repeated Algorithm 2 steps."""
    ins = _rand_instance(9, 7, 151)
    eta, k = 0.4 / math.sqrt(16), 192
    opts = ora.Options(tol=0.0, max_passes=k, check_every=64, adaptive_step=0, adaptive_restart=0,
                       primal_weight_update=0, beta=0.0, eta0=eta)
    res = ora.solve(ins.C, ins.f, ins.g, opts)
    assert res.status == ora.STATUS_MAX_ITER and res.restarts == 0 and res.candidate_is_average == 1
    X, p, q = np.zeros((9, 7)), np.zeros(9), np.zeros(7)
    Xs, ps, qs = [], [], []
    for _ in range(k):
        X, p, q = ora.pdhg_step(ins.C, ins.f, ins.g, X, p, q, eta, eta)
        Xs.append(X); ps.append(p); qs.append(q)
    np.testing.assert_allclose(res.X, np.mean(Xs, axis=0), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(res.p, np.mean(ps, axis=0), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(res.q, np.mean(qs, axis=0), rtol=1e-12, atol=1e-16)


def _constant_step_run(ora, ins, K, eta):
    """K constant-step Algorithm 2 iterations from the origin (pinned steps),
    with the uniform average and the KKT errors of both."""
    m, n = ins.C.shape
    X, p, q, Xb, pb, qb = ora.pdhg_steps(ins.C, ins.f, ins.g, np.zeros((m, n)), np.zeros(m), np.zeros(n),
                                        k=K, eta=eta)
    return (X, p, q), (Xb, pb, qb), ora.kkt(ins.C, ins.f, ins.g, X, p, q), ora.kkt(ins.C, ins.f, ins.g, Xb, pb, qb)


@pytest.mark.parametrize("K,average", [(1, True), (32, True), (64, False)])
def test_restart_candidate_is_the_lower_kkt_of_current_and_average(ora, K, average):
    """Sec. 5: the restart candidate is the current iterate if its KKT error is
    smaller than the running average's, else the average (reading C13: a tie,
    as after one step where both are the same point, goes to the average).
    With a constant step the solve's first check is reproduced from pinned
    Algorithm 2 steps; the three cases cover the tie and both outcomes."""
    ins = _rand_instance(9, 7, 161)
    eta = 0.1
    cur, avg, kc, ka = _constant_step_run(ora, ins, K, eta)
    assert (kc.kkt == ka.kkt) == (K == 1) and (not kc.kkt < ka.kkt) == average
    res = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=0.0, max_passes=K, check_every=K, adaptive_step=0,
                                                     primal_weight_update=0, eta0=eta))
    assert res.candidate_is_average == int(average)
    for got, want in zip((res.X, res.p, res.q), avg if average else cur):
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("beta_art,max_passes,restarts", [(1.0, 640, 1), (0.5, 1280, 5)])
def test_artificial_restart_schedule(ora, beta_art, max_passes, restarts):
    """Sec. 5 condition (iii), k >= beta_art * total, with reading C8 (total
    counts the iterations since the solve began, k those since the last
    restart, checks every 64 passes).  With (i) and (ii) switched off and a
    constant step every pass is accepted, so the schedule follows from the
    counts alone: beta_art = 1 restarts only at the first check; beta_art = 1/2
    restarts at passes 64, 128, 256, 512, 1024 (k doubles with total)."""
    ins = _rand_instance(9, 7, 162)
    res = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=0.0, max_passes=max_passes, adaptive_step=0,
                                                     beta_suff=0.0, beta_nec=0.0, beta_art=beta_art, eta0=0.1))
    assert res.status == ora.STATUS_MAX_ITER and res.rejected == 0 and res.iters == max_passes
    assert res.restarts == restarts


@pytest.mark.parametrize("theta", [0.0, 1.0])
def test_primal_weight_update_special_cases(ora, theta):
    """Sec. 5 PrimalWeightUpdate with smoothing theta at the one restart of a
    constant-step run (beta_art = 1, pass 64, candidate = current iterate, as
    in the K = 64 case above): theta = 0 keeps omega = 1; theta = 1 makes omega
    the ratio of the dual to the primal distance moved since the start."""
    ins = _rand_instance(9, 7, 161)
    (X, p, q), _, kc, ka = _constant_step_run(ora, ins, 64, 0.1)
    assert kc.kkt < ka.kkt
    res = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=0.0, max_passes=128, adaptive_step=0, beta_suff=0.0,
                                                     beta_nec=0.0, beta_art=1.0, eta0=0.1, theta=theta))
    assert res.restarts == 1
    want = 1.0 if theta == 0.0 else math.sqrt(p @ p + q @ q) / np.linalg.norm(X)
    assert abs(res.omega - want) <= 1e-13 * want


def test_adaptive_default_step_is_one_over_norm_A(ora):
    """Reading C2: the adaptive mode starts from eta0 = 1 / ||A||_2 = 1 / sqrt(m + n)
    (Prop. 1): the default run and a run given that eta0 are the same run."""
    ins = _rand_instance(20, 12, 163)
    a = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=1e-6))
    b = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=1e-6, eta0=1.0 / math.sqrt(32)))
    assert (a.passes, a.restarts, a.rejected) == (b.passes, b.restarts, b.rejected)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.p, b.p) and a.eta == b.eta


# --------------------------------------------------------------------------
# Sec. 5 adaptive step size (reading C6, PDLP's rule), on instances small
# enough to take one step by hand
# --------------------------------------------------------------------------
#
# With m = n = 1 (or m = 2, n = 1) one Algorithm 2 step is a handful of
# scalar operations, so eta_bar, the accept/reject decision and the next step
# size follow from the rule's statement without the oracle's code:
#   eta_bar = (omega ||dX||^2 + ||(dp, dq)||^2 / omega) / (2 |dp^T dX 1 + dq^T dX^T 1|),
#   accept iff eta <= eta_bar,  eta' = min((1 - t^-0.3) eta_bar, (1 + t^-0.6) eta)
# with t = 2 + (iterations accepted so far); eta' is used next either way.

def _few_passes(ora, C, f, g, X0, p0, q0, eta0, omega0, passes=1):
    """A solve stopped by its pass budget after `passes` passes (one check,
    at the end), adaptive step on, primal-weight update off."""
    opts = ora.Options(tol=0.0, max_passes=passes, check_every=passes, adaptive_step=1, primal_weight_update=0,
                       eta0=eta0, omega0=omega0)
    arr = lambda v: np.array(v, dtype=np.float64)  # noqa: E731
    return ora.solve(arr(C), arr(f), arr(g), opts, X0=arr(X0), p0=arr(p0), q0=arr(q0))


@pytest.mark.parametrize("case", STEP_RULE_CASES, ids=lambda c: c["name"])
def test_step_rule_one_pass_by_hand(ora, case):
    """One pass of the adaptive step-size rule on a 1 x 1 or 2 x 1 instance
    whose eta_bar and decision are derived by hand (tests/heuristic_cases.py):
    a rejection that keeps the state, an acceptance with omega = 2 (tests where
    omega enters eta_bar), and a rejection that needs the column part of
    dy^T A dx and of ||dy||^2."""
    r = _few_passes(ora, case["C"], case["f"], case["g"], case["X0"], case["p0"], case["q0"], case["eta0"],
                    case["omega0"])
    assert (r.passes, r.iters, r.rejected) == (1, case["iters"], case["rejected"])
    assert abs(r.eta - case["eta"]) <= 1e-15
    assert np.array_equal(r.X, np.array(case["X"])) and np.array_equal(r.p, np.array(case["p"]))
    assert np.array_equal(r.q, np.array(case["q"]))


def test_step_rule_grows_the_step_while_the_plan_does_not_move(ora):
    """1 x 1, C = 1, f = g = 1 from the origin with eta = 0.3: the first two
    passes leave X = 0 (reduced cost C - p - q = 1, then 1 - 0.6 = 0.4 > 0),
    so dX = 0, dy^T A dx = 0, eta_bar = +inf: both are accepted and the step
    grows by (1 + t^-0.6) with t = 2, then t = 3."""
    r = _few_passes(ora, [[1.0]], [1.0], [1.0], [[0.0]], [0.0], [0.0], 0.3, 1.0, passes=2)
    assert (r.passes, r.iters, r.rejected) == (2, 2, 0)
    assert r.X[0, 0] == 0.0
    assert abs(r.eta - 0.3 * (1 + 2 ** -0.6) * (1 + 3 ** -0.6)) <= 1e-15


def test_step_rule_from_the_origin_grows_then_rejects(ora):
    (C, f, g), eta2 = step_rule_from_origin_case()
    r = _few_passes(ora, C, f, g, [[0.0]], [0.0], [0.0], 1.0, 1.0, passes=2)
    assert (r.passes, r.iters, r.rejected) == (2, 1, 1)
    assert r.X[0, 0] == 0.0 and r.p[0] == 1.0 and r.q[0] == 1.0
    assert abs(r.eta - eta2) <= 1e-15 * eta2


# --------------------------------------------------------------------------
# Sec. 5 restart conditions (i) and (ii), each alone, with a constant step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["i", "ii"])
def test_restart_condition_alone(ora, which):
    """Each of Sec. 5's conditions (i) and (ii) alone (the others switched
    off: beta_nec = 0 or beta_suff = 0, and beta_art so large that (iii) never
    holds), constant step 0.1, a check every 8 passes.  A solve whose pass
    budget ends at check j (where its termination test comes first) has not
    restarted; one whose budget ends a check later restarted once, at check j,
    to that check's candidate, and returns the candidate of the next 8 steps."""
    ins, opts, j, want = restart_condition_case(ora, which)
    K = opts["check_every"]
    assert (which, j) in (("i", 3), ("ii", 4))
    r0 = ora.solve(ins.C, ins.f, ins.g, ora.Options(max_passes=j * K, **opts))
    assert r0.status == ora.STATUS_MAX_ITER and r0.restarts == 0
    r1 = ora.solve(ins.C, ins.f, ins.g, ora.Options(max_passes=(j + 1) * K, **opts))
    assert r1.status == ora.STATUS_MAX_ITER and r1.restarts == 1
    for got, w in zip((r1.X, r1.p, r1.q), want):
        np.testing.assert_allclose(got, w, rtol=1e-12, atol=1e-16)


def test_solve_rel_mode_one_plus(ora):
    """Reading C5, option 1 (cuPDLP's '1 +' denominators) also terminates correctly."""
    ins = I.points_instance(30, 30, 121)
    res = ora.solve(ins.C, ins.f, ins.g, ora.Options(tol=1e-6, rel_mode=1))
    k = ora.kkt(ins.C, ins.f, ins.g, res.X, res.p, res.q, rel_mode=1)
    assert res.status == 0 and k.rel_kkt <= 1e-6
    assert abs(k.rel_kkt - res.rel_kkt) < 1e-15


# --------------------------------------------------------------------------
# Algorithm 3 and Lemma 2
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [131, 132, 133])
def test_rounding_feasible_and_lemma2(ora, seed):
    rng = np.random.default_rng(seed)
    m, n = 13, 17
    f, g = rng.dirichlet(np.ones(m)), rng.dirichlet(np.ones(n))
    X = np.outer(f, g) * rng.uniform(0.5, 1.5, (m, n))
    Xf = ora.round_plan(X, f, g)
    assert Xf.min() >= 0.0
    np.testing.assert_allclose(Xf.sum(1), f, atol=1e-15)
    np.testing.assert_allclose(Xf.sum(0), g, atol=1e-15)
    viol = np.abs(f - X.sum(1)).sum() + np.abs(g - X.sum(0)).sum()
    assert np.abs(Xf - X).sum() <= 2.0 * viol + 1e-15


def test_rounding_keeps_feasible_plan(ora):
    ins = I.points_instance(6, 9, 141)
    obj, X, p, q = ora.exact_transport(ins.C, ins.f, ins.g)
    np.testing.assert_allclose(ora.round_plan(X, ins.f, ins.g), X, atol=1e-16)


def test_rounding_closed_forms(ora):
    """Algorithm 3 on two families with a closed-form result.  P is a feasible
    plan.  (a) alpha P, 0 < alpha < 1: every row and column is short, both
    scales are capped at 1, and the rank-one correction adds the missing mass
    (1 - alpha) f g^T.  (b) diag(d) P with d >= 1: the row step alone restores
    P, after which the columns are exact and nothing else changes."""
    ins = I.points_instance(7, 11, 142, marginals="dirichlet")
    f, g = ins.f, ins.g
    _, P, _, _ = ora.exact_transport(ins.C, f, g)
    P = 0.5 * P + 0.5 * np.outer(f, g)     # dense: every row and column carries mass
    for alpha in (0.25, 0.9):
        np.testing.assert_allclose(ora.round_plan(alpha * P, f, g), alpha * P + (1 - alpha) * np.outer(f, g),
                                   rtol=1e-13, atol=1e-17)
    d = np.random.default_rng(143).uniform(1.0, 3.0, 7)
    np.testing.assert_allclose(ora.round_plan(d[:, None] * P, f, g), P, rtol=1e-13, atol=1e-17)


# --------------------------------------------------------------------------
# Sec. 5.1: costs defined from point (pixel) coordinates
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 8])
def test_points_cost_matches_scipy_cdist(ora, d):
    """The cost-on-the-fly input, C_ij = dist(x_i, y_j) / divisor, against
    scipy's pairwise-distance routine for each distance the paper uses."""
    cdist = pytest.importorskip("scipy.spatial.distance").cdist
    rng = np.random.default_rng(100 + d)
    xs, ys = rng.random((13, d)), rng.random((9, d))
    for dist, metric in [("sqeuclid", "sqeuclidean"), ("l1", "cityblock"), ("l2", "euclidean"),
                         ("linf", "chebyshev")]:
        np.testing.assert_allclose(ora.points_cost(xs, ys, dist, 3.0), cdist(xs, ys, metric) / 3.0,
                                   rtol=1e-14, atol=1e-16)


def test_points_cost_grid_invariants(ora):
    """Pixel grid against itself: symmetric, zero diagonal, integer squared
    distances before scaling, and l_inf <= l2 <= l1 <= d l_inf, sqeuclid = l2^2."""
    G = 6
    P = np.array([(a, b) for a in range(G) for b in range(G)], dtype=np.float64)
    sq = ora.points_cost(P, P, "sqeuclid")
    l1, l2, li = (ora.points_cost(P, P, k) for k in ("l1", "l2", "linf"))
    assert np.array_equal(sq, sq.T) and not np.any(np.diag(sq))
    assert np.array_equal(sq, np.round(sq)) and sq.max() == 2 * (G - 1) ** 2
    assert np.all(li <= l2 + 1e-15) and np.all(l2 <= l1 + 1e-15) and np.all(l1 <= 2 * li + 1e-15)
    np.testing.assert_allclose(l2 ** 2, sq, rtol=1e-14, atol=1e-14)
    # the corner-to-corner distances
    assert l1[0, -1] == 2 * (G - 1) and li[0, -1] == G - 1


def test_points_cost_rejects_bad_arguments(ora):
    with pytest.raises(ValueError):
        ora.points_cost(np.zeros((2, 2)), np.zeros((2, 2)), "l1", 0.0)


# --------------------------------------------------------------------------
# Weak-duality lower bound of Eq. (1) from a row dual
# --------------------------------------------------------------------------

def test_dual_bound_single_row_is_the_optimum_for_any_p(ora):
    """One source: the only feasible plan is X = g^T, so OPT = C g, and for
    any p the bound p f + sum_j g_j (C_j - p) = C g (Sigma g = f) is exact.
    Hand case: C = [1, 3], f = 1, g = [1/2, 1/2], p = 1/4: q = [3/4, 11/4],
    bound 1/4 + 3/8 + 11/8 = 2 = OPT."""
    C = np.array([[1.0, 3.0]])
    lower, q = ora.dual_bound(C, np.array([1.0]), np.array([0.5, 0.5]), np.array([0.25]))
    np.testing.assert_array_equal(q, [0.75, 2.75])
    assert lower == 2.0
    rng = np.random.default_rng(7)
    C = rng.random((1, 9))
    g = rng.dirichlet(np.ones(9))
    for p0 in (-3.0, 0.0, 0.4, 17.0):
        lower, _ = ora.dual_bound(C, np.array([1.0]), g, np.array([p0]))
        assert abs(lower - C[0] @ g) <= 1e-14 * (1.0 + abs(p0))


@pytest.mark.parametrize("m,n,seed", [(12, 9, 141), (30, 41, 142), (64, 64, I.seed_for(0))])
def test_dual_bound_is_tight_at_the_exact_duals(ora, m, n, seed):
    """Strong duality: at the exact solver's optimal duals (p*, q*), q*_j <=
    min_i (C_ij - p*_i), so the bound is >= f^T p* + g^T q* = OPT and, by weak
    duality, equal to it; the column dual it forms is >= q*."""
    ins = I.points_instance(m, n, seed)
    opt, _, ps, qs = ora.exact_transport(ins.C, ins.f, ins.g)
    lower, q = ora.dual_bound(ins.C, ins.f, ins.g, ps)
    assert abs(lower - opt) <= 1e-12 * opt
    assert np.all(q >= qs - 1e-14)
    # feasible: p*_i + q_j <= C_ij, with equality somewhere in every column
    slack = ins.C - ps[:, None] - q[None, :]
    assert slack.min() >= 0.0 and np.all(slack.min(axis=0) == 0.0)


def test_dual_bound_below_the_optimum_and_shift_invariant(ora):
    """Weak duality for arbitrary p (the bound never exceeds OPT), and a
    shift p + c moves q by -c and leaves the bound unchanged (Sigma f =
    Sigma g)."""
    ins = I.points_instance(23, 31, 143)
    opt, *_ = ora.exact_transport(ins.C, ins.f, ins.g)
    rng = np.random.default_rng(8)
    for _ in range(5):
        p = rng.standard_normal(23)
        lower, q = ora.dual_bound(ins.C, ins.f, ins.g, p)
        assert lower <= opt + 1e-15
        l2, q2 = ora.dual_bound(ins.C, ins.f, ins.g, p + 0.375)
        np.testing.assert_allclose(q2, q - 0.375, rtol=0, atol=1e-15)
        assert abs(l2 - lower) <= 1e-14
