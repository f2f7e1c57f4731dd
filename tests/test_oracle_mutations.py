"""Mutation check of the oracle's pins.

Each case plants one plausible mistake (a dropped term, a wrong sign, a
swapped step size, an off-by-one weight) in a copy of ``oracle/pdot_oracle.c``,
builds it on the CPU, and runs ``tests/test_oracle_pins.py`` against it in a
child process; at least one pin must fail.  No mistake changes an index or a
buffer size, so every mutant stays memory-safe.

The Sec. 5 heuristics are pinned through special cases where their outcome
follows from pinned steps and counts (the candidate rule, the artificial
restart schedule, the primal weight at theta = 0 and 1, the default first
step, restart conditions (i) and (ii) each alone) and through one-step cases
of the step-size rule derived by hand (reading C6).  For the mutants of the
step-size rule and of conditions (i) and (ii) the check also names the pin
that must fail: a direct pin, not only an end-to-end solve.
"""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pdot_oracle.c")

# (id, text in the oracle, planted replacement)
MUTANTS = [
    ("At_sign", "Y[i * n + j] = p[i] + q[j];", "Y[i * n + j] = p[i] - q[j];"),
    ("A_column_drops_row0", "c[j] += X[i * n + j];", "c[j] += X[i * n + j] * (double)(i > 0);"),
    ("step_reduced_cost_sign", "double v = X[e] - tau * (C[e] - AtY[e]);",
     "double v = X[e] - tau * (C[e] + AtY[e]);"),
    ("step_no_projection", "Xn[e] = v > 0.0 ? v : 0.0;", "Xn[e] = v;"),
    ("step_no_extrapolation", "E[e] = 2.0 * Xn[e] - X[e];", "E[e] = Xn[e];"),
    ("step_p_uses_tau", "pn[i] = p[i] + sigma * (f[i] - rE[i]);", "pn[i] = p[i] + tau * (f[i] - rE[i]);"),
    ("step_q_sign", "qn[j] = q[j] + sigma * (g[j] - cE[j]);", "qn[j] = q[j] - sigma * (g[j] - cE[j]);"),
    ("kkt_drops_gap", "out->kkt = sqrt(rp2 + rd2 + (out->gap / R) * (out->gap / R));",
     "out->kkt = sqrt(rp2 + rd2);"),
    ("kkt_dual_residual_sign", "double v = p[i] + q[j] - C[i * n + j];", "double v = C[i * n + j] - p[i] - q[j];"),
    ("kkt_drops_column_residual", "for (int64_t j = 0; j < n; ++j) rp2 += (c[j] - g[j]) * (c[j] - g[j]);", ";"),
    ("kkt_rel_d_wrong_scale", "out->rel_d = sqrt(rd2) / den_d;", "out->rel_d = sqrt(rd2) / den_p;"),
    ("kkt_rel_gap_drops_dual", "den_g = fabs(cx) + fabs(dual);", "den_g = fabs(cx);"),
    ("solve_norm_C_squared", "norm_C = sqrt(norm_C);", ";"),
    ("average_weight_off_by_one", "wn = 1.0 / (double)(k + 1);", "wn = 1.0 / (double)(k + 2);"),
    ("round_no_rank_one", "if (l1 > 0.0)", "if (l1 < 0.0)"),
    ("round_row_scale_uncapped", "if (xi > 1.0) xi = 1.0;", ";"),
    ("round_stale_column_sums", "ora_apply_A(m, n, Xf, r, c);\n    for (int64_t j = 0; j < n; ++j) {\n        double yj",
     "for (int64_t j = 0; j < n; ++j) {\n        double yj"),
    ("exact_reverse_arc_cost_sign", "double rcost = -C[i * n + j] + pi[u] - pi[i];",
     "double rcost = C[i * n + j] + pi[u] - pi[i];"),
    ("exact_dual_sign", "p[i] = -pi[i];", "p[i] = pi[i];"),
    ("exact_ignores_reverse_capacity", "if (cap < delta) delta = cap;", ";"),
    ("points_sqrt_on_sqeuclid", "if (kind == 2) acc = sqrt(acc);", "if (kind == 0 || kind == 2) acc = sqrt(acc);"),
    ("points_linf_sums", "else if (fabs(t) > acc) acc = fabs(t);", "else acc += fabs(t);"),
    ("theory_step_too_large", "0.5 / sqrt((double)(m + n))", "1.0 / sqrt((double)(m + n))"),
    ("kkt_gap_sign", "out->gap = cx - dual;", "out->gap = dual - cx;"),
    ("round_error_sign", "r[i] = f[i] - r[i];", "r[i] = r[i] - f[i];"),
    ("exact_potential_update", "pi[v] += (dist[v] < dt ? dist[v] : dt);", "pi[v] += (dist[v] < dt ? dist[v] : 0.0);"),
    ("points_divisor_ignored", "C[i * n + j] = acc / divisor;", "C[i * n + j] = acc;"),
    ("restart_kkt0_not_updated", "        kkt0 = kk->kkt;\n        kkt_prev = kk->kkt;\n        k = 0;",
     "        kkt_prev = kk->kkt;\n        k = 0;"),
    ("candidate_tie_inverted", "use_avg = !(kc.kkt < ka.kkt);", "use_avg = (kc.kkt < ka.kkt);"),
    ("restart_sufficient_flipped", "restart = (kk->kkt <= opt->beta_suff * kkt0)",
     "restart = (kk->kkt >= opt->beta_suff * kkt0)", "restart_condition_alone"),
    ("restart_artificial_dropped", "|| ((double)k >= opt->beta_art * (double)total);", ";"),
    ("eta_bar_drops_factor_two", "(2.0 * fabs(inter))", "(fabs(inter))", "step_rule"),
    ("eta_growth_exponent", "pow(t1, -0.6)", "pow(t1, -0.3)", "step_rule"),
    ("eta_bar_omega_swapped", "(omega * dX2 + dy2 / omega)", "(dX2 / omega + omega * dy2)", "step_rule"),
    ("eta_inter_drops_columns", "inter += (qn[j] - q[j]) * cd[j];", ";", "step_rule"),
    ("eta_dy_drops_columns", "dy2 += (qn[j] - q[j]) * (qn[j] - q[j]);", ";", "step_rule"),
    ("eta_schedule_index", "double t1 = (double)(total + 2);", "double t1 = (double)(total + 3);", "step_rule"),
    ("eta_accept_after_update", "accept = eta <= eta_bar;", "accept = eta_next <= eta_bar;", "step_rule"),
    ("eta_shrink_uses_eta", "double a = (1.0 - pow(t1, -0.3)) * eta_bar;", "double a = (1.0 - pow(t1, -0.3)) * eta;",
     "step_rule"),
    ("restart_sufficient_vs_previous", "restart = (kk->kkt <= opt->beta_suff * kkt0)",
     "restart = (kk->kkt <= opt->beta_suff * kkt_prev)", "restart_condition_alone"),
    ("restart_necessary_no_rise_test", "(kk->kkt <= opt->beta_nec * kkt0 && kk->kkt > kkt_prev)",
     "(kk->kkt <= opt->beta_nec * kkt0)", "restart_condition_alone"),
    ("restart_necessary_rise_vs_start", "&& kk->kkt > kkt_prev)", "&& kk->kkt > kkt0)", "restart_condition_alone"),
    ("restart_previous_not_tracked", "            kkt_prev = kk->kkt;\n            continue;", "            continue;",
     "restart_condition_alone"),
    ("primal_weight_inverted", "log(dy / dX)", "log(dX / dy)"),
    ("adaptive_eta0_doubled", "eta = opt->adaptive_step ? 1.0 / sqrt", "eta = opt->adaptive_step ? 2.0 / sqrt"),
    ("dual_bound_max_not_min", "if (v < q_out[j]) q_out[j] = v;", "if (v > q_out[j]) q_out[j] = v;", "dual_bound"),
    ("dual_bound_adds_p", "double v = C[i * n + j] - p[i];", "double v = C[i * n + j] + p[i];", "dual_bound"),
    ("dual_bound_skips_row1", "for (int64_t i = 1; i < m; ++i) {\n        for (int64_t j = 0; j < n; ++j) {\n            double v = C[i * n + j] - p[i];",
     "for (int64_t i = 2; i < m; ++i) {\n        for (int64_t j = 0; j < n; ++j) {\n            double v = C[i * n + j] - p[i];",
     "dual_bound"),
    ("dual_bound_drops_f_term", "for (int64_t i = 0; i < m; ++i) s += f[i] * p[i];", ";", "dual_bound"),
]


def _failed_pins(out: str):
    return sorted(set(re.findall(r"FAILED \S*::(\S+)", out)))


@pytest.mark.parametrize("case", MUTANTS, ids=lambda c: c[0])
def test_pins_catch_planted_mistake(tmp_path, case):
    name, old, new = case[:3]
    direct = case[3] if len(case) > 3 else None   # a pin that must fail by itself
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} is not unique"
    base = str(tmp_path / "oracle_mutant")
    with open(base + ".c", "w") as fh:
        fh.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", base + ".so", base + ".c", "-lm"])
    env = dict(os.environ, PDOT_ORACLE_MUTANT=base)
    pins = os.path.join(ROOT, "tests", "test_oracle_pins.py")
    args = [pins, "-x"] if direct is None else [pins, "-k", direct]
    r = subprocess.run([sys.executable, "-m", "pytest", *args, "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode in (0, 1), out[-2000:]
    assert r.returncode == 1, f"mutant {name} survived every pin" + ("" if direct is None else f" named {direct!r}")
    assert _failed_pins(out), out[-2000:]
