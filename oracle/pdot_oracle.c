/*
 * pdot_oracle.c -- plain, slow, FP64 CPU oracle for PDOT (restarted PDHG for
 * discrete optimal transport, arXiv 2407.19689).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is FP64, row-major (X[i*n + j], i < m rows, j < n columns), with
 * plain loops in the order the paper writes the steps.  No blocking, fusion or
 * reordering beyond what each definition states.
 *
 * Contents and the passage each function follows:
 *   ora_apply_A / ora_apply_At   Eq. (4) and the implicit products in Sec. 3.1:
 *                                A vec(X) = [X 1_n ; X^T 1_m],
 *                                A^T [p;q] = p 1_n^T + 1_m q^T.
 *   ora_pdhg_step                one inner iteration of Algorithm 2
 *                                (primal projection, then the two dual updates
 *                                that use the extrapolated plan 2X^+ - X).
 *   ora_lp_pdhg_step             one inner iteration of Algorithm 1 on a generic
 *                                standard-form LP with an explicit dense A.
 *   ora_kkt                      KKT error of the OT problem (Sec. 3.1, the
 *                                display after Algorithm 2) and the relative
 *                                termination measures (reading C5).
 *   ora_solve                    Algorithm 2 with the enhancements of Sec. 5:
 *                                adaptive restarts (three conditions), adaptive
 *                                step size (PDLP rule, reading C6), primal-weight
 *                                update; or the fixed-beta restart of Eq. (6)
 *                                with a constant step (theory mode).
 *   ora_round                    Algorithm 3 (rounding onto the feasible set).
 *   ora_exact_transport          exact optimum of Eq. (1) by successive shortest
 *                                paths with node potentials (not in the paper:
 *                                the plain definition of the LP optimum).
 *   ora_dual_bound               a lower bound on the optimum of Eq. (1) from
 *                                any row dual p: the dual of Eq. (1) asks
 *                                p_i + q_j <= C_ij (the constraint whose
 *                                violation the KKT error's dual term measures,
 *                                Sec. 3.1), and the largest q it allows for a
 *                                given p is q_j = min_i (C_ij - p_i); weak
 *                                duality then gives f^T p + g^T q <= OPT (not
 *                                in the paper: the plain definition).
 *   ora_points_cost              C_ij = dist(x_i, y_j) / divisor for the
 *                                distances the paper's grid costs use (Sec. 5.1:
 *                                l1, l2, l_inf; squared l2 for the squared grid
 *                                distance), the input of cost-on-the-fly solves.
 *
 * Readings of passages the paper leaves open are listed beside the code that
 * takes them, numbered C1..C16.
 * The adaptive heuristics are pinned by special cases (restart candidate
 * rule, artificial-restart schedule, restart conditions (i) and (ii) each
 * alone, primal weight at theta = 0 and 1, default first step), by one-step
 * cases of the step-size rule derived by hand on 1 x 1 and 2 x 1 instances,
 * and end to end (the solve reaches the exact optimum).  The paper prints no
 * trajectory, so the sequence of decisions along a real solve is pinned only
 * through these cases and end to end.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_MAX_ITER 5
#define ORA_ERR_ARG 1
#define ORA_ERR_NUMERIC 4

/* ------------------------------------------------------------------------- */
/* Eq. (4): implicit products with the constraint matrix A.                   */
/* ------------------------------------------------------------------------- */

/* r = X 1_n (row sums), c = X^T 1_m (column sums). */
void ora_apply_A(int64_t m, int64_t n, const double *X, double *r, double *c)
{
    for (int64_t i = 0; i < m; ++i) r[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            r[i] += X[i * n + j];
            c[j] += X[i * n + j];
        }
    }
}

/* Y = p 1_n^T + 1_m q^T. */
void ora_apply_At(int64_t m, int64_t n, const double *p, const double *q, double *Y)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            Y[i * n + j] = p[i] + q[j];
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2, one inner iteration (tau = primal step, sigma = dual step).   */
/*   X+ = Proj_{R+}(X - tau (C - p 1^T - 1 q^T))                              */
/*   p+ = p + sigma (f - (2X+ - X) 1)                                         */
/*   q+ = q + sigma (g - (2X+ - X)^T 1)                                       */
/* ------------------------------------------------------------------------- */
void ora_pdhg_step(int64_t m, int64_t n, const double *C, const double *f, const double *g,
                   const double *X, const double *p, const double *q, double tau, double sigma,
                   double *Xn, double *pn, double *qn)
{
    double *AtY = (double *)malloc(sizeof(double) * (size_t)(m * n));
    double *E = (double *)malloc(sizeof(double) * (size_t)(m * n));
    double *rE = (double *)malloc(sizeof(double) * (size_t)m);
    double *cE = (double *)malloc(sizeof(double) * (size_t)n);

    ora_apply_At(m, n, p, q, AtY);
    for (int64_t e = 0; e < m * n; ++e) {
        double v = X[e] - tau * (C[e] - AtY[e]);
        Xn[e] = v > 0.0 ? v : 0.0;
    }
    for (int64_t e = 0; e < m * n; ++e) E[e] = 2.0 * Xn[e] - X[e];
    ora_apply_A(m, n, E, rE, cE);
    for (int64_t i = 0; i < m; ++i) pn[i] = p[i] + sigma * (f[i] - rE[i]);
    for (int64_t j = 0; j < n; ++j) qn[j] = q[j] + sigma * (g[j] - cE[j]);

    free(AtY); free(E); free(rE); free(cE);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1, one inner iteration on min c^T x s.t. Ax = b, x >= 0 with an  */
/* explicit dense A (M x N, row-major).                                        */
/*   x+ = Proj(x - eta (c - A^T y)),  y+ = y + sigma (b - A(2x+ - x))          */
/* ------------------------------------------------------------------------- */
void ora_lp_pdhg_step(int64_t M, int64_t N, const double *A, const double *b, const double *c,
                      const double *x, const double *y, double eta, double sigma,
                      double *xn, double *yn)
{
    for (int64_t k = 0; k < N; ++k) {
        double aty = 0.0;
        for (int64_t r = 0; r < M; ++r) aty += A[r * N + k] * y[r];
        double v = x[k] - eta * (c[k] - aty);
        xn[k] = v > 0.0 ? v : 0.0;
    }
    for (int64_t r = 0; r < M; ++r) {
        double ax = 0.0;
        for (int64_t k = 0; k < N; ++k) ax += A[r * N + k] * (2.0 * xn[k] - x[k]);
        yn[r] = y[r] + sigma * (b[r] - ax);
    }
}

/* ------------------------------------------------------------------------- */
/* KKT error of the OT problem (Sec. 3.1):                                     */
/*   KKT^2 = ||X1 - f||^2 + ||X^T1 - g||^2 + ||[p1^T + 1q^T - C]^+||_F^2       */
/*           + ((<C,X> - f^T p - g^T q) / R)^2                                 */
/* Relative measures (reading C5; the paper uses "relative KKT error" for its  */
/* termination test without defining it).  rel_mode 0 (default) divides each  */
/* part by the size of the data it is measured against:                        */
/*   rel_p   = ||[X1 - f; X^T1 - g]|| / ||[f;g]||                              */
/*   rel_d   = ||[p1^T + 1q^T - C]^+||_F / ||C||_F                             */
/*   rel_gap = |<C,X> - f^T p - g^T q| / (|<C,X>| + |f^T p + g^T q|)            */
/* rel_mode 1 uses the cuPDLP denominators 1 + ||[f;g]||, 1 + ||C||_F and      */
/* 1 + |<C,X>| + |f^T p + g^T q|.  A zero denominator is replaced by 1.        */
/*   rel_kkt = max(rel_p, rel_d, rel_gap)                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double rp2;      /* ||X1 - f||^2 + ||X^T1 - g||^2 */
    double rd2;      /* ||[p1^T + 1q^T - C]^+||_F^2 */
    double cx;       /* <C, X> */
    double dual;     /* f^T p + g^T q */
    double gap;      /* cx - dual */
    double kkt;      /* KKT error as printed (R-scaled gap) */
    double rel_p, rel_d, rel_gap, rel_kkt;
} ora_kkt_t;

void ora_kkt(int64_t m, int64_t n, const double *C, const double *f, const double *g,
             const double *X, const double *p, const double *q, double R,
             double norm_b, double norm_C, int rel_mode, ora_kkt_t *out)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    ora_apply_A(m, n, X, r, c);

    double rp2 = 0.0;
    for (int64_t i = 0; i < m; ++i) rp2 += (r[i] - f[i]) * (r[i] - f[i]);
    for (int64_t j = 0; j < n; ++j) rp2 += (c[j] - g[j]) * (c[j] - g[j]);

    double rd2 = 0.0, cx = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double v = p[i] + q[j] - C[i * n + j];
            if (v > 0.0) rd2 += v * v;
            cx += C[i * n + j] * X[i * n + j];
        }
    }
    double dual = 0.0;
    for (int64_t i = 0; i < m; ++i) dual += f[i] * p[i];
    for (int64_t j = 0; j < n; ++j) dual += g[j] * q[j];

    out->rp2 = rp2;
    out->rd2 = rd2;
    out->cx = cx;
    out->dual = dual;
    out->gap = cx - dual;
    out->kkt = sqrt(rp2 + rd2 + (out->gap / R) * (out->gap / R));
    double den_p = norm_b, den_d = norm_C, den_g = fabs(cx) + fabs(dual);
    if (rel_mode == 1) { den_p += 1.0; den_d += 1.0; den_g += 1.0; }
    if (den_p <= 0.0) den_p = 1.0;
    if (den_d <= 0.0) den_d = 1.0;
    if (den_g <= 0.0) den_g = 1.0;
    out->rel_p = sqrt(rp2) / den_p;
    out->rel_d = sqrt(rd2) / den_d;
    out->rel_gap = fabs(out->gap) / den_g;
    out->rel_kkt = out->rel_p;
    if (out->rel_d > out->rel_kkt) out->rel_kkt = out->rel_d;
    if (out->rel_gap > out->rel_kkt) out->rel_kkt = out->rel_gap;
    free(r); free(c);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 with the Sec. 5 enhancements.                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    double tol;               /* relative KKT tolerance (termination) */
    int64_t max_passes;       /* bound on PDHG passes (accepted + rejected) */
    int64_t check_every;      /* restart/termination check after every K-th pass (C8) */
    int adaptive_step;        /* 1: PDLP step rule (C6); 0: constant eta */
    int adaptive_restart;     /* 1: three conditions of Sec. 5; 0: fixed beta, Eq. (6) */
    int primal_weight_update; /* 1: PrimalWeightUpdate at restarts (Sec. 5) */
    double beta;              /* fixed-beta restart decay (theory mode) */
    double beta_suff, beta_nec, beta_art;
    double theta;             /* primal-weight smoothing */
    double eta0;              /* initial (or constant) step; <= 0 picks the default (C2) */
    double omega0;            /* initial primal weight (C11) */
    double R;                 /* gap scaling in KKT (C3) */
    double eps_zero;          /* C10 */
    int rel_mode;             /* C5: 0 scale-relative, 1 cuPDLP "1 +" denominators */
} ora_options;

typedef struct {
    int status;
    double primal_obj, dual_obj, gap, kkt;
    double rel_p, rel_d, rel_gap, rel_kkt;
    int64_t iters, passes, restarts, rejected;
    double eta, omega;
    int candidate_is_average;
} ora_result;

static double ora_sqdist(int64_t len, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t e = 0; e < len; ++e) s += (a[e] - b[e]) * (a[e] - b[e]);
    return s;
}

static void ora_fill_result(ora_result *res, const ora_kkt_t *k)
{
    res->primal_obj = k->cx;
    res->dual_obj = k->dual;
    res->gap = k->gap;
    res->kkt = k->kkt;
    res->rel_p = k->rel_p;
    res->rel_d = k->rel_d;
    res->rel_gap = k->rel_gap;
    res->rel_kkt = k->rel_kkt;
}

/*
 * Solve Eq. (1).  On entry X (m*n), p (m), q (n) hold the initial point (C1:
 * callers pass zeros for the default start).  On exit they hold the returned
 * iterate: the restart candidate that met the tolerance (or the candidate of
 * the last check when the pass budget ran out).
 */
int ora_solve(int64_t m, int64_t n, const double *C, const double *f, const double *g,
              const ora_options *opt, double *X, double *p, double *q, ora_result *res)
{
    const int64_t mn = m * n;
    memset(res, 0, sizeof(*res));
    if (m < 1 || n < 1 || opt->check_every < 1) { res->status = ORA_ERR_ARG; return ORA_ERR_ARG; }

    double norm_b = 0.0;
    for (int64_t i = 0; i < m; ++i) norm_b += f[i] * f[i];
    for (int64_t j = 0; j < n; ++j) norm_b += g[j] * g[j];
    norm_b = sqrt(norm_b);
    double norm_C = 0.0;
    for (int64_t e = 0; e < mn; ++e) norm_C += C[e] * C[e];
    norm_C = sqrt(norm_C);

    double *Xn = (double *)malloc(sizeof(double) * (size_t)mn);
    double *Xb = (double *)malloc(sizeof(double) * (size_t)mn);
    double *Xa = (double *)malloc(sizeof(double) * (size_t)mn);   /* restart anchor X^{t,0} */
    double *pn = (double *)malloc(sizeof(double) * (size_t)m);
    double *pb = (double *)malloc(sizeof(double) * (size_t)m);
    double *pa = (double *)malloc(sizeof(double) * (size_t)m);
    double *qn = (double *)malloc(sizeof(double) * (size_t)n);
    double *qb = (double *)malloc(sizeof(double) * (size_t)n);
    double *qa = (double *)malloc(sizeof(double) * (size_t)n);
    double *rd = (double *)malloc(sizeof(double) * (size_t)m);     /* (X+ - X) 1 */
    double *cd = (double *)malloc(sizeof(double) * (size_t)n);     /* (X+ - X)^T 1 */
    double *D = (double *)malloc(sizeof(double) * (size_t)mn);

    /* Step sizes (C2): adaptive mode starts at 1/||A||_2 = 1/sqrt(m+n)
     * (Proposition 1); the constant-step (theory) mode uses 1/(2 sqrt(m+n)),
     * the bound of Theorems 1 and 2. */
    double eta = opt->eta0;
    if (eta <= 0.0) eta = opt->adaptive_step ? 1.0 / sqrt((double)(m + n)) : 0.5 / sqrt((double)(m + n));
    double omega = opt->omega0 > 0.0 ? opt->omega0 : 1.0;

    int64_t k = 0, total = 0, passes = 0, restarts = 0, rejected = 0;
    ora_kkt_t kc, ka;
    memcpy(Xa, X, sizeof(double) * (size_t)mn);
    memcpy(pa, p, sizeof(double) * (size_t)m);
    memcpy(qa, q, sizeof(double) * (size_t)n);
    ora_kkt(m, n, C, f, g, X, p, q, opt->R, norm_b, norm_C, opt->rel_mode, &kc);
    double kkt0 = kc.kkt, kkt_prev = kc.kkt;
    int status = -1;
    if (kc.rel_kkt <= opt->tol) {
        ora_fill_result(res, &kc);
        status = ORA_OK;
    }

    while (status < 0) {
        double tau = eta / omega, sigma = eta * omega;
        ora_pdhg_step(m, n, C, f, g, X, p, q, tau, sigma, Xn, pn, qn);
        passes++;

        int accept = 1;
        if (opt->adaptive_step) {
            /* Step-size test of Sec. 5 in the PDLP form (reading C6):
             *   eta_bar = (omega ||dX||^2 + ||(dp,dq)||^2 / omega) / (2 |dp^T dX 1 + dq^T dX^T 1|)
             *   eta'    = min((1 - (t+1)^-0.3) eta_bar, (1 + (t+1)^-0.6) eta),
             * t = 1-based index of the iteration being attempted (accepted so far + 1),
             * so the first factor is never 0.  eta_bar = +inf when the denominator is 0.
             * The step is accepted when eta <= eta_bar; eta' is used next either way. */
            for (int64_t e = 0; e < mn; ++e) D[e] = Xn[e] - X[e];
            ora_apply_A(m, n, D, rd, cd);
            double dX2 = 0.0, dy2 = 0.0, inter = 0.0;
            for (int64_t e = 0; e < mn; ++e) dX2 += D[e] * D[e];
            for (int64_t i = 0; i < m; ++i) { dy2 += (pn[i] - p[i]) * (pn[i] - p[i]); inter += (pn[i] - p[i]) * rd[i]; }
            for (int64_t j = 0; j < n; ++j) { dy2 += (qn[j] - q[j]) * (qn[j] - q[j]); inter += (qn[j] - q[j]) * cd[j]; }
            double eta_bar = inter != 0.0 ? (omega * dX2 + dy2 / omega) / (2.0 * fabs(inter)) : INFINITY;
            double t1 = (double)(total + 2);
            double a = (1.0 - pow(t1, -0.3)) * eta_bar;
            double b = (1.0 + pow(t1, -0.6)) * eta;
            double eta_next = a < b ? a : b;
            accept = eta <= eta_bar;
            eta = eta_next;
        }

        if (accept) {
            memcpy(X, Xn, sizeof(double) * (size_t)mn);
            memcpy(p, pn, sizeof(double) * (size_t)m);
            memcpy(q, qn, sizeof(double) * (size_t)n);
            /* Running average with uniform weights (Algorithm 2, C7). */
            double wo = (double)k / (double)(k + 1), wn = 1.0 / (double)(k + 1);
            if (k == 0) {
                memcpy(Xb, X, sizeof(double) * (size_t)mn);
                memcpy(pb, p, sizeof(double) * (size_t)m);
                memcpy(qb, q, sizeof(double) * (size_t)n);
            } else {
                for (int64_t e = 0; e < mn; ++e) Xb[e] = wo * Xb[e] + wn * X[e];
                for (int64_t i = 0; i < m; ++i) pb[i] = wo * pb[i] + wn * p[i];
                for (int64_t j = 0; j < n; ++j) qb[j] = wo * qb[j] + wn * q[j];
            }
            k++;
            total++;
        } else {
            rejected++;
        }

        if (passes % opt->check_every != 0) continue;

        if (k == 0) {
            /* No accepted step since the last restart: nothing new to evaluate. */
            if (passes >= opt->max_passes) {
                ora_kkt(m, n, C, f, g, X, p, q, opt->R, norm_b, norm_C, opt->rel_mode, &kc);
                ora_fill_result(res, &kc);
                status = ORA_MAX_ITER;
            }
            continue;
        }

        /* Restart candidate (Sec. 5): the current iterate if its KKT error is
         * strictly smaller than the average's, else the average (C13). */
        ora_kkt(m, n, C, f, g, X, p, q, opt->R, norm_b, norm_C, opt->rel_mode, &kc);
        ora_kkt(m, n, C, f, g, Xb, pb, qb, opt->R, norm_b, norm_C, opt->rel_mode, &ka);
        if (!isfinite(kc.kkt) || !isfinite(ka.kkt)) { status = ORA_ERR_NUMERIC; ora_fill_result(res, &kc); break; }
        int use_avg;
        if (opt->adaptive_restart) use_avg = !(kc.kkt < ka.kkt);
        else use_avg = 1;   /* Algorithm 2 / Eq. (6): restart to the average */
        const ora_kkt_t *kk = use_avg ? &ka : &kc;
        double *Xc = use_avg ? Xb : X, *pc = use_avg ? pb : p, *qc = use_avg ? qb : q;

        if (kk->rel_kkt <= opt->tol || passes >= opt->max_passes) {
            ora_fill_result(res, kk);
            res->candidate_is_average = use_avg;
            if (use_avg) {
                memcpy(X, Xb, sizeof(double) * (size_t)mn);
                memcpy(p, pb, sizeof(double) * (size_t)m);
                memcpy(q, qb, sizeof(double) * (size_t)n);
            }
            status = kk->rel_kkt <= opt->tol ? ORA_OK : ORA_MAX_ITER;
            break;
        }

        int restart;
        if (opt->adaptive_restart) {
            restart = (kk->kkt <= opt->beta_suff * kkt0)
                   || (kk->kkt <= opt->beta_nec * kkt0 && kk->kkt > kkt_prev)
                   || ((double)k >= opt->beta_art * (double)total);
        } else {
            restart = ka.kkt <= opt->beta * kkt0;
        }

        if (!restart) {
            kkt_prev = kk->kkt;
            continue;
        }

        /* PrimalWeightUpdate (Sec. 5) between the new restart point and the previous one. */
        if (opt->primal_weight_update) {
            double dX = sqrt(ora_sqdist(mn, Xc, Xa));
            double dy = sqrt(ora_sqdist(m, pc, pa) + ora_sqdist(n, qc, qa));
            if (dX > opt->eps_zero && dy > opt->eps_zero)
                omega = exp(opt->theta * log(dy / dX) + (1.0 - opt->theta) * log(omega));
        }
        if (use_avg) {
            memcpy(X, Xb, sizeof(double) * (size_t)mn);
            memcpy(p, pb, sizeof(double) * (size_t)m);
            memcpy(q, qb, sizeof(double) * (size_t)n);
        }
        memcpy(Xa, X, sizeof(double) * (size_t)mn);
        memcpy(pa, p, sizeof(double) * (size_t)m);
        memcpy(qa, q, sizeof(double) * (size_t)n);
        kkt0 = kk->kkt;
        kkt_prev = kk->kkt;
        k = 0;
        restarts++;
    }

    res->status = status;
    res->iters = total;
    res->passes = passes;
    res->restarts = restarts;
    res->rejected = rejected;
    res->eta = eta;
    res->omega = omega;

    free(Xn); free(Xb); free(Xa); free(pn); free(pb); free(pa);
    free(qn); free(qb); free(qa); free(rd); free(cd); free(D);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3: rounding onto {X >= 0, X1 = f, X^T1 = g}.                      */
/* Guards (C12): a row or column whose sum is 0 keeps scale 1; when            */
/* ||err_r||_1 = 0 the rank-one correction is skipped.                         */
/* ------------------------------------------------------------------------- */
void ora_round(int64_t m, int64_t n, const double *X, const double *f, const double *g, double *Xf)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    ora_apply_A(m, n, X, r, c);
    for (int64_t i = 0; i < m; ++i) {
        double xi = r[i] > 0.0 ? f[i] / r[i] : 1.0;
        if (xi > 1.0) xi = 1.0;
        for (int64_t j = 0; j < n; ++j) Xf[i * n + j] = xi * X[i * n + j];
    }
    ora_apply_A(m, n, Xf, r, c);
    for (int64_t j = 0; j < n; ++j) {
        double yj = c[j] > 0.0 ? g[j] / c[j] : 1.0;
        if (yj > 1.0) yj = 1.0;
        for (int64_t i = 0; i < m; ++i) Xf[i * n + j] *= yj;
    }
    ora_apply_A(m, n, Xf, r, c);
    double l1 = 0.0;
    for (int64_t i = 0; i < m; ++i) { r[i] = f[i] - r[i]; l1 += fabs(r[i]); }
    for (int64_t j = 0; j < n; ++j) c[j] = g[j] - c[j];
    if (l1 > 0.0)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j) Xf[i * n + j] += r[i] * c[j] / l1;
    free(r); free(c);
}

/* ------------------------------------------------------------------------- */
/* Exact optimum of Eq. (1): successive shortest paths with node potentials.   */
/* Sources i carry supply f_i, sinks j demand g_j, arcs i->j cost C_ij with    */
/* unbounded capacity; the residual reverse arc j->i (cost -C_ij) has capacity */
/* X_ij.  Dijkstra over reduced costs C_ij + pi_i - pi_j >= 0 (dense, O(V^2)). */
/* Returns the plan, the duals p_i = -pi_i, q_j = pi_j (so p_i + q_j <= C_ij   */
/* with equality where X_ij > 0) and the objective.                            */
/* ------------------------------------------------------------------------- */
int ora_exact_transport(int64_t m, int64_t n, const double *C, const double *f, const double *g,
                        double *X, double *p, double *q, double *obj)
{
    const int64_t V = m + n;          /* nodes 0..m-1 sources, m..m+n-1 sinks */
    double *pi = (double *)calloc((size_t)V, sizeof(double));
    double *dist = (double *)malloc(sizeof(double) * (size_t)V);
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    char *done = (char *)malloc((size_t)V);
    double *sup = (double *)malloc(sizeof(double) * (size_t)m);
    double *dem = (double *)malloc(sizeof(double) * (size_t)n);
    double total = 0.0, total_g = 0.0;
    for (int64_t i = 0; i < m; ++i) { sup[i] = f[i]; total += f[i]; }
    for (int64_t j = 0; j < n; ++j) { dem[j] = g[j]; total_g += g[j]; }
    if (total_g > total) total = total_g;
    const double eps = 1e-15 * (total > 0.0 ? total : 1.0);
    for (int64_t e = 0; e < m * n; ++e) X[e] = 0.0;
    /* Feasible start for the potentials: pi_sink(j) = min_i C_ij keeps every
     * forward reduced cost non-negative. */
    for (int64_t j = 0; j < n; ++j) {
        double mn_ = INFINITY;
        for (int64_t i = 0; i < m; ++i) if (C[i * n + j] < mn_) mn_ = C[i * n + j];
        pi[m + j] = mn_;
    }

    int rc = ORA_OK;
    for (int64_t guard = 0;; ++guard) {
        int any_sup = 0, any_dem = 0;
        for (int64_t i = 0; i < m; ++i) if (sup[i] > eps) { any_sup = 1; break; }
        for (int64_t j = 0; j < n; ++j) if (dem[j] > eps) { any_dem = 1; break; }
        if (!any_sup || !any_dem) break;
        if (guard > 100 * (V + 10) * (V + 10)) { rc = ORA_ERR_NUMERIC; break; }

        for (int64_t v = 0; v < V; ++v) { dist[v] = INFINITY; prev[v] = -1; done[v] = 0; }
        for (int64_t i = 0; i < m; ++i) if (sup[i] > eps) dist[i] = 0.0;
        int64_t target = -1;
        for (;;) {
            int64_t u = -1;
            double du = INFINITY;
            for (int64_t v = 0; v < V; ++v) if (!done[v] && dist[v] < du) { du = dist[v]; u = v; }
            if (u < 0) break;
            done[u] = 1;
            if (u >= m && dem[u - m] > eps) { target = u; break; }
            if (u < m) {
                for (int64_t j = 0; j < n; ++j) {
                    int64_t v = m + j;
                    if (done[v]) continue;
                    double rcost = C[u * n + j] + pi[u] - pi[v];
                    if (rcost < 0.0) rcost = 0.0;   /* clamp rounding below zero */
                    if (du + rcost < dist[v]) { dist[v] = du + rcost; prev[v] = u; }
                }
            } else {
                int64_t j = u - m;
                for (int64_t i = 0; i < m; ++i) {
                    if (done[i] || X[i * n + j] <= 0.0) continue;
                    double rcost = -C[i * n + j] + pi[u] - pi[i];
                    if (rcost < 0.0) rcost = 0.0;
                    if (du + rcost < dist[i]) { dist[i] = du + rcost; prev[i] = u; }
                }
            }
        }
        if (target < 0) { rc = ORA_ERR_NUMERIC; break; }
        const double dt = dist[target];
        for (int64_t v = 0; v < V; ++v) pi[v] += (dist[v] < dt ? dist[v] : dt);

        /* Bottleneck of the path: source supply, sink demand, reverse-arc flows. */
        double delta = dem[target - m];
        int64_t v = target;
        while (prev[v] >= 0) {
            int64_t u = prev[v];
            if (u >= m) {  /* reverse arc sink u -> source v carries X[v][u-m] */
                double cap = X[v * n + (u - m)];
                if (cap < delta) delta = cap;
            }
            v = u;
        }
        if (sup[v] < delta) delta = sup[v];
        int64_t s = v;
        v = target;
        while (prev[v] >= 0) {
            int64_t u = prev[v];
            if (u < m) X[u * n + (v - m)] += delta;
            else X[v * n + (u - m)] -= delta;
            v = u;
        }
        sup[s] -= delta;
        dem[target - m] -= delta;
    }

    double o = 0.0;
    for (int64_t e = 0; e < m * n; ++e) o += C[e] * X[e];
    for (int64_t i = 0; i < m; ++i) p[i] = -pi[i];
    for (int64_t j = 0; j < n; ++j) q[j] = pi[m + j];
    *obj = o;
    free(pi); free(dist); free(prev); free(done); free(sup); free(dem);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Lower bound on the optimum from a row dual (weak duality of Eq. (1)).       */
/* ------------------------------------------------------------------------- */
/* q_out[j] = min over i of (C_ij - p_i), the largest column dual that keeps
 * p_i + q_j <= C_ij for every i; *lower = f^T p + g^T q_out.  Rows in order,
 * then the two dot products in order. */
void ora_dual_bound(int64_t m, int64_t n, const double *C, const double *f, const double *g,
                    const double *p, double *q_out, double *lower)
{
    for (int64_t j = 0; j < n; ++j) q_out[j] = C[j] - p[0];
    for (int64_t i = 1; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double v = C[i * n + j] - p[i];
            if (v < q_out[j]) q_out[j] = v;
        }
    }
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += f[i] * p[i];
    for (int64_t j = 0; j < n; ++j) s += g[j] * q_out[j];
    *lower = s;
}

/* ------------------------------------------------------------------------- */
/* Cost matrix from point coordinates (Sec. 5.1 defines the grid costs as      */
/* distances between pixel coordinates).  xs is m x d, ys is n x d, row-major. */
/* kind: 0 squared Euclidean, 1 l1, 2 l2 (Euclidean), 3 l_inf.                 */
/* C_ij = dist(x_i, y_j) / divisor, every step in FP64.                        */
/* ------------------------------------------------------------------------- */
int ora_points_cost(int64_t m, int64_t n, int d, const double *xs, const double *ys, int kind, double divisor,
                    double *C)
{
    if (d < 1 || kind < 0 || kind > 3 || !(divisor > 0.0)) return ORA_ERR_ARG;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = xs[i * d + k] - ys[j * d + k];
                if (kind == 0 || kind == 2) acc += t * t;
                else if (kind == 1) acc += fabs(t);
                else if (fabs(t) > acc) acc = fabs(t);
            }
            if (kind == 2) acc = sqrt(acc);
            C[i * n + j] = acc / divisor;
        }
    }
    return ORA_OK;
}
