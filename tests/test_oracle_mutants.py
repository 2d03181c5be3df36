"""The oracle's pins catch plausible slips.

Each case copies ``oracle/pps_oracle.c`` to a temporary directory, plants
one mistake of the kind a careful reader could still make (a dropped
factor, a flipped sign, a transposed operand, an off-by-one index, a wrong
comparison), builds that copy with gcc and runs the pin checks of
test_oracle_pins.py against it.  At least one pin must fail for every
mutant.  Nothing here touches the real oracle or any GPU.
"""
from __future__ import annotations

import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_dpps as dpps_pins
from tests import test_oracle_run as run_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "pps_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("ball: dropped factor 2", "double disc = v * v - 2.0 * a * s;",
     "double disc = v * v - a * s;"),
    ("ball: wrong root", "return 2.0 * s / (v + sqrt(disc));",
     "return (v + sqrt(disc)) / a;"),
    ("intercept: sign in projection", "double w = (ux * dx + uy * dy) / d;",
     "double w = (ux * dx - uy * dy) / d;"),
    ("intercept: projection onto o - p", "double w = (ux * dx + uy * dy) / d;",
     "double w = -(ux * dx + uy * dy) / d;"),
    ("intercept: clamp dropped", "if (w > vmax) w = vmax;", ";"),
    ("intercept: d_top missing 2",
     "double d_top = (vmax * vmax - w * w) / (2.0 * amax);",
     "double d_top = (vmax * vmax - w * w) / amax;"),
    ("intercept: cruise term dropped",
     "return t_top + (dist - d_top) / vmax;", "return t_top + dist / vmax;"),
    ("intercept: reach ignored in distance", "double dist = d - reach;",
     "double dist = d;"),
    ("intercept: accel root sign",
     "return (-w + sqrt(w * w + 2.0 * amax * dist)) / amax;",
     "return (w + sqrt(w * w + 2.0 * amax * dist)) / amax;"),
    ("min over opponents flipped", "if (t < T) T = t;", "if (t > T) T = t;"),
    ("sample: transposed operand", "double px = bx + f * (cx - bx);",
     "double px = bx + f * (cy - by);"),
    ("sample: off-by-one index", "double f = (double)k / (double)K;",
     "double f = (double)(k - 1) / (double)K;"),
    ("sample: ball distance not scaled", "double s = f * D;",
     "double s = D;"),
    ("margin: operands swapped", "double diff = T - tb;",
     "double diff = tb - T;"),
    ("reachability: dropped factor 2",
     "int reach_ok = (v * v - 2.0 * a * D >= 0.0);",
     "int reach_ok = (v * v - a * D >= 0.0);"),
    ("shot: atan for asin", "double half = asin(r / d);",
     "double half = atan(r / d);"),
    ("shot: sweep forgets nesting", "if (e[i] > cur) cur = e[i];",
     "cur = e[i];"),
    ("shot: lower post sign", "double lo = atan2(-hw - cy, gx - cx);",
     "double lo = atan2(-hw + cy, gx - cx);"),
    ("shot: goal at the far edge", "double gx = 0.5 * st->sc[PPS_ORACLE_FIELD_LEN];",
     "double gx = st->sc[PPS_ORACLE_FIELD_LEN];"),
    ("score: distance sign", "- prm[PPS_ORACLE_W_DIST] * dist_goal / diag",
     "+ prm[PPS_ORACLE_W_DIST] * dist_goal / diag"),
    ("score: goal point", "double gdx = 0.5 * L - cx, gdy = 0.0 - cy;",
     "double gdx = L - cx, gdy = 0.0 - cy;"),
    ("score: cap ignored", "? margin\n                      : prm[PPS_ORACLE_MARGIN_CAP];",
     "? margin\n                      : margin;"),
    ("argmax: ties to the larger index", "(sc == bs && idx < bi)",
     "(sc == bs && idx > bi)"),
    ("grid: edge excluded", "*nx = (int)lround(L / g) + 1;",
     "*nx = (int)lround(L / g);"),
]

CHECKS = [pins.check_hand_ball, pins.check_hand_intercept,
          pins.check_hand_shot, pins.check_hand_score, pins.check_hand_grid,
          pins.check_invariants, pins.check_shot_closed_form,
          pins.check_score_closed_form, pins.check_search_tie_rule,
          pins.check_search_reachability, pins.check_search_consistency,
          pins.check_ball_vs_sim, pins.check_intercept_vs_sim,
          pins.check_margin_vs_sim, pins.check_shot_vs_rays,
          pins.check_intercept_monotone]


# Running points (Sec. 5.1-5.2), checked by the running-point pins.
RUN_MUTANTS = [
    ("run: zone cut at L/2", "return (px >= 0.25 * L - tol ? 2 : 0) + (py >= ys - tol ? 1 : 0);",
     "return (px >= 0.5 * L - tol ? 2 : 0) + (py >= ys - tol ? 1 : 0);"),
    ("run: no edge tolerance", "return prm[PPS_ORACLE_R_SPACING] / 1024.0;",
     "return 0.0;"),
    ("run: zone ignores the ball", "double ys = by < -0.25 * W ? -0.25 * W : (by > 0.25 * W ? 0.25 * W : by);",
     "double ys = 0.0;"),
    ("run: zone clamp dropped", "double ys = by < -0.25 * W ? -0.25 * W : (by > 0.25 * W ? 0.25 * W : by);",
     "double ys = by;"),
    ("run: goal distance over L", "double x_goal = sqrt(gx * gx + gy * gy) / sqrt(L * L + W * W);",
     "double x_goal = sqrt(gx * gx + gy * gy) / L;"),
    ("run: ball credit uncapped", "double x_ball = (db < ref ? db : ref) / ref;",
     "double x_ball = db / ref;"),
    ("run: angle band low side dropped", "double off = alpha < lo ? lo - alpha : (alpha > hi ? alpha - hi : 0.0);",
     "double off = alpha > hi ? alpha - hi : 0.0;"),
    ("run: angle credit not clamped", "double x_angle = 1.0 - (f > 1.0 ? 1.0 : f);",
     "double x_angle = 1.0 - f;"),
    ("run: both lines to one post", "side ? hw : -hw", "hw"),
    ("run: guards outside the area", "if (o[0] < x0 || o[0] > x1 || o[1] < y0 || o[1] > y1) continue;",
     ";"),
    ("run: slowest guard", "if (t < T) T = t;\n            }\n        }\n        tsum += T;",
     "if (t > T || T == cap) T = t;\n            }\n        }\n        tsum += T;"),
    ("run: guard cap not applied", "double ex, ey, T = cap;", "double ex, ey, T = 1e300;"),
    ("run: entry at the far side", "*ex = px + t0 * dx;\n    *ey = py + t0 * dy;",
     "*ex = px + t1 * dx;\n    *ey = py + t1 * dy;"),
    ("run: avoid comparison flipped", "if (dj < db) x_avoid = 1.0;",
     "if (dj > db) x_avoid = 1.0;"),
    ("run: avoid sign", "- prm[PPS_ORACLE_R_W_AVOID] * x_avoid",
     "+ prm[PPS_ORACLE_R_W_AVOID] * x_avoid"),
    ("run: goal sign", "cand ? -prm[PPS_ORACLE_R_W_GOAL] * x_goal",
     "cand ? prm[PPS_ORACLE_R_W_GOAL] * x_goal"),
    ("run: defence area kept", "int cand = !(px > x0 + tol && py > y0 + tol && py < y1 - tol);",
     "int cand = 1;"),
    ("run: ties to the larger index", "if (out[7] != 0.0 && (bi[z] < 0 || out[0] > bs[z])) {",
     "if (out[7] != 0.0 && (bi[z] < 0 || out[0] >= bs[z])) {"),
    ("run: back pair first", "for (int pair = 1; pair >= 0; --pair) {",
     "for (int pair = 0; pair <= 1; ++pair) {"),
    ("run: pass zone not avoided", "best_idx[z] >= 0 && z != avoid", "best_idx[z] >= 0"),
    ("run: grid y from 0", "double py = fmin(-0.5 * W + j * g, 0.5 * W);",
     "double py = fmin(j * g, 0.5 * W);"),
]


# The direction x power search, passing power and shooting (Sec. 4.1-4.4),
# checked by the pins of the direction x power search.
DPPS_MUTANTS = [
    ("dpps: wrong field edge", "if (ux < 0.0) s_out = fmin(s_out, (-hl - bx) / ux);",
     "if (ux < 0.0) s_out = fmin(s_out, (hl - bx) / ux);"),
    ("dpps: stop distance missing 2", "double s_stop = v * v / (2.0 * a);",
     "double s_stop = v * v / a;"),
    ("dpps: ball at rest at 2v/a", "double tk = last_stop ? v / a : pps_oracle_ball_time(s, v, a);",
     "double tk = last_stop ? 2.0 * v / a : pps_oracle_ball_time(s, v, a);"),
    ("dpps: stop sample ignores the robot", "return T <= tk ? tk : T;", "return tk;"),
    ("dpps: samples start at the ball", "double s = (double)k / (double)K * S;",
     "double s = (double)(k - 1) / (double)K * S;"),
    ("dpps: group takes the slowest robot",
     "            if (t < T) {\n                T = t;\n                w = r;",
     "            if (t > T || w < 0) {\n                T = t;\n                w = r;"),
    ("dpps: no slide", "double v = prm[PPS_ORACLE_D_SLIDE] * v0;", "double v = v0;"),
    ("dpps: power grid over npow", "vlo + (double)j * (vhi - vlo) / (double)(npow - 1)",
     "vlo + (double)j * (vhi - vlo) / (double)npow"),
    ("dpps: half circle of directions", "double phi = 2.0 * pi * (double)i / (double)ndir;",
     "double phi = pi * (double)i / (double)ndir;"),
    ("dpps: delta sign", "(t_opp - t_team > prm[PPS_ORACLE_D_TAU_DELTA])",
     "(t_team - t_opp > prm[PPS_ORACLE_D_TAU_DELTA])"),
    ("dpps: refraction sign", "- prm[PPS_ORACLE_D_W_REFR] * refr / pi",
     "+ prm[PPS_ORACLE_D_W_REFR] * refr / pi"),
    ("dpps: delta uncapped", "(delta < cap ? delta : cap)", "delta"),
    ("dpps: refraction transposed", "double c = (ux * gx + uy * gy) / dg;",
     "double c = (ux * gx - uy * gy) / dg;"),
    ("dpps: receive point one sample short", "double s = (double)k_team / (double)st->K * S;",
     "double s = (double)(k_team - 1) / (double)st->K * S;"),
    ("pass: Eq. 1 sign", "double v1 = t > 0.0 ? (d + 0.5 * a * t * t) / t : INFINITY;",
     "double v1 = t > 0.0 ? (d - 0.5 * a * t * t) / t : INFINITY;"),
    ("pass: Eq. 2 inverted", "double v0 = v1 / slide;", "double v0 = v1 * slide;"),
    ("pass: buffer dropped", "double t = T + buffer;", "double t = T;"),
    ("shoot: aims at the gap's edge", "double dir = g0 + 0.5 * theta;",
     "double dir = g0 + theta;"),
    ("shoot: no slide", "double v = slide * v_shot;", "double v = v_shot;"),
    ("shoot: angle not required",
     "shoot = theta >= theta_min && (t_opp - t_line > tau || isinf(t_opp));",
     "shoot = (t_opp - t_line > tau || isinf(t_opp));"),
]


def _caught(orc, checks=None):
    for chk in checks or CHECKS:
        try:
            chk(orc)
        except (AssertionError, ValueError, ZeroDivisionError, OverflowError):
            return chk.__name__
    return None


@pytest.mark.parametrize("name,orig,mut", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert text.count(orig) >= 1, f"mutation site missing: {orig!r}"
    bad = os.path.join(tmp_path, "pps_oracle.c")
    with open(bad, "w") as f:
        f.write(text.replace(orig, mut, 1))
    shutil.copy(os.path.join(os.path.dirname(SRC), "pps_oracle.h"), tmp_path)
    lib = oracle.build(force=True, src=bad,
                       out=os.path.join(tmp_path, "libmutant.so"))
    caught = _caught(oracle.Oracle(lib))
    assert caught is not None, f"no pin caught mutant: {name}"


@pytest.mark.parametrize("name,orig,mut", RUN_MUTANTS,
                         ids=[m[0] for m in RUN_MUTANTS])
def test_running_point_mutant_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert text.count(orig) >= 1, f"mutation site missing: {orig!r}"
    bad = os.path.join(tmp_path, "pps_oracle.c")
    with open(bad, "w") as f:
        f.write(text.replace(orig, mut, 1))
    shutil.copy(os.path.join(os.path.dirname(SRC), "pps_oracle.h"), tmp_path)
    lib = oracle.build(force=True, src=bad,
                       out=os.path.join(tmp_path, "libmutant.so"))
    caught = _caught(oracle.Oracle(lib), run_pins.CHECKS)
    assert caught is not None, f"no pin caught mutant: {name}"


@pytest.mark.parametrize("name,orig,mut", DPPS_MUTANTS,
                         ids=[m[0] for m in DPPS_MUTANTS])
def test_direction_power_mutant_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert text.count(orig) >= 1, f"mutation site missing: {orig!r}"
    bad = os.path.join(tmp_path, "pps_oracle.c")
    with open(bad, "w") as f:
        f.write(text.replace(orig, mut, 1))
    shutil.copy(os.path.join(os.path.dirname(SRC), "pps_oracle.h"), tmp_path)
    lib = oracle.build(force=True, src=bad,
                       out=os.path.join(tmp_path, "libmutant.so"))
    caught = _caught(oracle.Oracle(lib), dpps_pins.CHECKS)
    assert caught is not None, f"no pin caught mutant: {name}"
