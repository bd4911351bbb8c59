"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one (the oracle's own source is never modified).

Each mutation is a dropped term, a wrong sign, a swapped index or operand, or
min/max confusion; the pin suite must fail on each mutated build.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sta_oracle.c")

MUTATIONS = {
    "late_max_becomes_min": ("if (v > best_at) best_at = v;", "if (v < best_at) best_at = v;"),
    "wire_delay_dropped": ("at[4 * p + q] = at[4 * d + q] + wd[p];", "at[4 * p + q] = at[4 * d + q];"),
    "unateness_ignored": ("int rfi = nl->arc_unate[OR_MAXA * t + ai] > 0 ? rf : 1 - rf;\n"
                          "                        size_t tab",
                          "int rfi = rf;\n                        size_t tab"),
    "no_slew_degradation": ("sl[4 * p + q] = sqrt(sl[4 * d + q] * sl[4 * d + q] + imp[p] * imp[p]);",
                            "sl[4 * p + q] = sl[4 * d + q];"),
    "driver_wire_cap_dropped": ("tcap[0] += 0.5 * cw * len;", ""),
    "table_axes_transposed": ("double t00 = tab[i * OR_LUT + j], t01 = tab[i * OR_LUT + j + 1];",
                              "double t00 = tab[j * OR_LUT + i], t01 = tab[i * OR_LUT + j + 1];"),
    "driver_gradient_sign": ("grad[2 * d] -= gd * sx;", "grad[2 * d] += gd * sx;"),
    "load_gradient_dropped": ("gload[p] += gD * dDl;", ""),
    "rat_adds_wire_delay": ("double v = rat[4 * s + q] - wd[s];", "double v = rat[4 * s + q] + wd[s];"),
    "early_rat_uses_min": ("if (q < 2) { if (v > rat[4 * p + q]) rat[4 * p + q] = v; }",
                           "if (q < 2) { if (v < rat[4 * p + q]) rat[4 * p + q] = v; }"),
    "lse_weight_sign": ("double w = exp((ats[2 * i + rfi] + D - ats[2 * p + rf]) / gamma);",
                        "double w = exp(-(ats[2 * i + rfi] + D - ats[2 * p + rf]) / gamma);"),
    "second_moment_factor": ("double m = 2.0 * beta[u] - delay[u] * delay[u];",
                             "double m = beta[u] - delay[u] * delay[u];"),
    "endpoint_slack_early_sign": ("double se = fmin(at[4 * p] - ce[0], at[4 * p + 1] - ce[1]);",
                                  "double se = fmin(ce[0] - at[4 * p], ce[1] - at[4 * p + 1]);"),
    "capture_adjoint_dropped": ("if (nl->end_clk && nl->end_clk[e] >= 0) gwd[nl->end_clk[e]] += dl_ds;", ""),
    "capture_edges_swapped": ("con[4 * e + q] += q < 2 ? at[4 * k + 2] : at[4 * k + 0];",
                              "con[4 * e + q] += q < 2 ? at[4 * k + 0] : at[4 * k + 2];"),
    "capture_arrival_subtracted": ("con[4 * e + q] += q < 2 ? at[4 * k + 2] : at[4 * k + 0];",
                                   "con[4 * e + q] -= q < 2 ? at[4 * k + 2] : at[4 * k + 0];"),
    # late output slew taken as the minimum over arcs, in the forward alone and
    # in the forward and the adjoint together (a consistent mistake)
    "late_slew_max_becomes_min": ("if (S > best_sl) { best_sl = S; argmax = ai; }",
                                  "if (argmax < 0 || S < best_sl) { best_sl = S; argmax = ai; }"),
    "late_slew_min_in_forward_and_adjoint": [
        ("if (S > best_sl) { best_sl = S; argmax = ai; }",
         "if (argmax < 0 || S < best_sl) { best_sl = S; argmax = ai; }"),
        ("if (S > best) { best = S; amax = a; dss = dSs; dsl = dSl; }",
         "if (amax < 0 || S < best) { best = S; amax = a; dss = dSs; dsl = dSl; }")],
    "late_slew_tie_to_last_arc": ("if (S > best) { best = S; amax = a; dss = dSs; dsl = dSl; }",
                                  "if (S >= best) { best = S; amax = a; dss = dSs; dsl = dSl; }"),
    # smoothed loss: the zero of the TNS soft-min dropped (loss and adjoint
    # alike), the soft-min's log term with the wrong sign, WNS over half the
    # slacks, rise and fall soft-minned separately
    "tns_softmin_drops_zero": [("tns_g += softmin(3, trip, gamma);", "tns_g += softmin(2, trip, gamma);"),
                               ("double te = softmin(3, trip, gamma);", "double te = softmin(2, trip, gamma);")],
    "softmin_log_sign": ("return m - gamma * log(s);", "return m + gamma * log(s);"),
    "wns_softmin_over_rise_only": ("double wns_g = softmin(2 * E, sm, gamma);",
                                   "double wns_g = softmin(E, sm, gamma);"),
    "tns_rise_fall_separately": ("tns_g += softmin(3, trip, gamma);",
                                 "{ double tr[2] = {sm[2 * e], 0.0}, tf[2] = {sm[2 * e + 1], 0.0};\n"
                                 "          tns_g += softmin(2, tr, gamma) + softmin(2, tf, gamma); }"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    edits = MUTATIONS[name]
    if isinstance(edits, tuple):
        edits = [edits]
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation anchor for {name} not unique"
        src = src.replace(old, new)
    mutated = tmp_path / "mut.c"
    mutated.write_text(src)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(mutated), "-lm"])
    env = dict(os.environ, ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_rc_nldm.py"),
                        os.path.join(ROOT, "tests", "test_oracle_sta.py"),
                        os.path.join(ROOT, "tests", "test_oracle_loss_slew.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pin suite"
