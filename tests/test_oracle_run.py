"""Pins of the oracle's running-point search (Sec. 5.1-5.2).

Each criterion against a closed form or a value worked out by hand, the
guard points P and Q against a brute-force walk along the line to the post,
the per-zone best against an argmax over the dense scores with the zones
recomputed here, the zone choice against hand cases, and mirror symmetry.
Each check takes an oracle build, so the mutant tests can run them against
copies with planted mistakes.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1909_07717_gb300 import synth

SC = {"ball_x": 0.0, "ball_y": 0.0, "ball_decel": 0.5, "vmax": 3.25,
      "amax": 3.0, "field_len": 12.0, "field_wid": 9.0, "goal_width": 1.8}
PRM = dict(spacing=0.1, w_goal=1.0, w_ball=1.0, w_angle=1.0, w_guard=1.0,
           w_avoid=1.0, ball_ref=2.0, angle_lo=0.25, angle_hi=0.75,
           angle_span=0.5, def_depth=1.2, def_width=2.4, guard_cap=2.0,
           n_run=4)


def _st(opp=(), ball=(0.0, 0.0)):
    sc = dict(SC, ball_x=ball[0], ball_y=ball[1])
    return oracle.DState(sc, np.zeros((0, 4)),
                         np.array(opp, float).reshape(-1, 4), 1)


def _from_rest(d, vmax=3.25, amax=3.0):
    if d <= vmax * vmax / (2 * amax):
        return math.sqrt(2 * d / amax)
    return d / vmax + vmax / (2 * amax)


def check_zones_split_at_quarter_length_and_the_ball(orc):
    st = _st()
    assert [orc.run_zone(st, p) for p in
            ((1, -4), (1, 4), (5, -4), (5, 4))] == [0, 1, 2, 3]
    assert orc.run_zone(st, (3.0, 0.0)) == 3      # both cuts inclusive
    assert orc.run_zone(st, (2.99, -0.01)) == 0
    # the cut follows the ball's y, but stays within +-W/4 = 2.25
    up = _st(ball=(0.0, 1.5))
    assert orc.run_zone(up, (1, 1.4)) == 0
    assert orc.run_zone(up, (1, 1.6)) == 1
    far = _st(ball=(-3.0, 4.0))
    assert orc.run_zone(far, (1, 2.2)) == 0
    assert orc.run_zone(far, (1, 2.3)) == 1
    # outside the attacking half there is no zone
    assert orc.run_zone(st, (-0.1, 0.0)) == -1
    assert orc.run_zone(st, (6.1, 0.0)) == -1
    assert orc.run_zone(st, (3.0, 4.6)) == -1


def check_distance_criteria_and_the_defence_area(orc):
    st = _st(ball=(1.0, 0.0))
    r = orc.run_point(st, PRM, (0.0, 0.0))
    assert math.isclose(r["goal"], 6.0 / 15.0, rel_tol=1e-14)  # diag 15
    assert math.isclose(r["ball"], 0.5, rel_tol=1e-14)         # 1 m of 2
    r = orc.run_point(st, PRM, (4.0, 3.0))
    assert math.isclose(r["goal"], math.hypot(2.0, 3.0) / 15.0,
                        rel_tol=1e-14)
    assert r["ball"] == 1.0                                    # beyond 2 m
    # the interior of the defence area (x > 4.8, |y| < 1.2) holds no
    # candidate; its boundary does
    r = orc.run_point(st, PRM, (5.5, 0.0))
    assert not r["candidate"] and r["score"] == -math.inf
    for p in ((5.5, 1.2), (4.8, 0.0), (5.5, -1.3)):
        assert orc.run_point(st, PRM, p)["candidate"], p


def check_angle_credit_is_a_band_off_the_goal_axis(orc):
    st = _st()
    for alpha, want in ((0.0, 0.5), (0.25, 1.0), (0.5, 1.0), (0.75, 1.0),
                        (1.0, 0.5), (1.25, 0.0), (1.4, 0.0)):
        d = 3.0
        p = (6.0 - d * math.cos(alpha), d * math.sin(alpha))
        r = orc.run_point(st, PRM, p)
        assert math.isclose(r["angle"], want, abs_tol=1e-12), (alpha, r)
        q = orc.run_point(st, PRM, (p[0], -p[1]))
        assert math.isclose(q["angle"], want, abs_tol=1e-12)


def _entry(p, post, x0=4.8, x1=6.0, y1=1.2, steps=200000):
    """First point of the segment p -> post inside the defence area, by
    walking along it."""
    for k in range(steps + 1):
        t = k / steps
        x = p[0] + t * (post[0] - p[0])
        y = p[1] + t * (post[1] - p[1])
        if x0 <= x <= x1 and -y1 <= y <= y1:
            return x, y
    return None


def check_guard_time_to_p_and_q_against_a_walk_along_the_lines(orc):
    rng = np.random.default_rng(3)
    for _ in range(40):
        p = (rng.uniform(0, 4.7), rng.uniform(-4.5, 4.5))
        g = (rng.uniform(4.8, 6.0), rng.uniform(-1.2, 1.2))
        st = _st(opp=[(g[0], g[1], 0.0, 0.0)])
        r = orc.run_point(st, PRM, p)
        tot = 0.0
        for post in ((6.0, -0.9), (6.0, 0.9)):
            e = _entry(p, post)
            assert e is not None          # the line ends at a post inside
            tot += min(_from_rest(math.dist(e, g)), 2.0)
        assert math.isclose(r["guard"], tot / 4.0, abs_tol=2e-4), (p, g, r)
    # a line entering through the side of the area: p = (5.5, 3), post
    # (6, 0.9) crosses y = 1.2 at x = 5.5 + 0.5 * 1.8 / 2.1; a guard at rest
    # there takes no time to P
    px = 5.5 + 0.5 * 1.8 / 2.1
    st = _st(opp=[(px, 1.2, 0.0, 0.0)])
    r = orc.run_point(st, PRM, (5.5, 3.0))
    q = _entry((5.5, 3.0), (6.0, -0.9))
    want = (0.0 + min(_from_rest(math.dist(q, (px, 1.2))), 2.0)) / 4.0
    assert math.isclose(r["guard"], want, abs_tol=2e-4)


def check_guards_are_only_the_opponents_inside_the_area(orc):
    # no opponent at all, or only opponents outside the area: the cap
    assert orc.run_point(_st(), PRM, (3.0, 1.0))["guard"] == 1.0
    st = _st(opp=[(4.7, 0.0, 0.0, 0.0), (6.1, 0.0, 0.0, 0.0)])
    assert orc.run_point(st, PRM, (3.0, 1.0))["guard"] == 1.0
    # the faster of two guards counts, per point
    a = _st(opp=[(5.9, 0.0, 0.0, 0.0)])
    b = _st(opp=[(5.9, 0.0, 0.0, 0.0), (4.9, 0.3, 0.0, 0.0)])
    ga = orc.run_point(a, PRM, (3.0, 1.0))["guard"]
    gb = orc.run_point(b, PRM, (3.0, 1.0))["guard"]
    assert gb < ga


def check_avoid_is_set_when_an_opponent_is_nearer_the_ball(orc):
    st = _st(opp=[(2.0, 0.0, 0.0, 0.0)], ball=(1.0, 0.0))
    assert orc.run_point(st, PRM, (1.5, 0.0))["avoid"] == 0.0  # 0.5 < 1
    assert orc.run_point(st, PRM, (3.0, 0.0))["avoid"] == 1.0  # 2 > 1
    assert orc.run_point(_st(), PRM, (3.0, 0.0))["avoid"] == 0.0


def check_score_is_the_weighted_sum_with_costs_signed(orc):
    st = _st(opp=[(5.5, 0.2, 0.5, -0.3), (0.5, 0.5, 0.0, 0.0)],
             ball=(1.0, 0.0))
    w = dict(w_goal=0.7, w_ball=1.3, w_angle=0.4, w_guard=2.0, w_avoid=0.9)
    r = orc.run_point(st, dict(PRM, **w), (3.3, -2.1))
    assert r["avoid"] == 1.0 and 0 < r["guard"] < 1
    want = (-0.7 * r["goal"] + 1.3 * r["ball"] + 0.4 * r["angle"]
            + 2.0 * r["guard"] - 0.9 * r["avoid"])
    assert math.isclose(r["score"], want, rel_tol=1e-14)
    # with one weight at a time the score is that criterion (signed)
    for k, crit, sign in (("w_goal", "goal", -1), ("w_ball", "ball", 1),
                          ("w_angle", "angle", 1), ("w_guard", "guard", 1),
                          ("w_avoid", "avoid", -1)):
        one = dict(PRM, w_goal=0.0, w_ball=0.0, w_angle=0.0, w_guard=0.0,
                   w_avoid=0.0)
        one[k] = 1.0
        r1 = orc.run_point(st, one, (3.3, -2.1))
        assert r1["score"] == sign * r1[crit]


def _zones_here(batch, s, nx, ny, g):
    """The zone of every grid point, computed here from the definition."""
    L = float(batch["field_len"][s])
    W = float(batch["field_wid"][s])
    by = float(batch["ball"][s][1])
    ys = min(max(by, -W / 4), W / 4)
    x = np.minimum(np.arange(nx) * g, L / 2)
    y = np.minimum(-W / 2 + np.arange(ny) * g, W / 2)
    X, Y = np.meshgrid(x, y)
    return (X >= L / 4) * 2 + (Y >= ys)


def check_best_per_zone_is_the_argmax_of_the_dense_scores(orc):
    batch = synth.run_states(11, 6)
    prm = synth.run_oracle_params()
    r = orc.run_search(batch, prm, dense=True)
    g = prm["spacing"]
    ny, nx = r["score"].shape[1:]
    assert (nx, ny) == (61, 91)
    for s in range(6):
        z = _zones_here(batch, s, nx, ny, g).reshape(-1)
        sc = r["score"][s].reshape(-1)
        for q in range(4):
            cand = np.where((z == q) & np.isfinite(sc))[0]
            i = cand[np.argmax(sc[cand])]     # the first of equal maxima
            assert r["best_idx"][s, q] == i
            assert r["best_score"][s, q] == sc[i]
        assert np.isinf(sc).sum() > 0         # the defence area's interior


def check_ties_go_to_the_lowest_index(orc):
    """All weights 0: every candidate ties, so each zone's best is its
    first grid point (in j * nx + i order)."""
    batch = synth.run_states(14, 2)
    prm = dict(synth.run_oracle_params(), w_goal=0.0, w_ball=0.0,
               w_angle=0.0, w_guard=0.0, w_avoid=0.0)
    r = orc.run_search(batch, prm, dense=True)
    ny, nx = r["score"].shape[1:]
    for s in range(2):
        z = _zones_here(batch, s, nx, ny, prm["spacing"]).reshape(-1)
        for q in range(4):
            assert r["best_idx"][s, q] == np.where(z == q)[0][0]
            assert r["best_score"][s, q] == 0.0


def check_raster_ends_on_the_goal_and_touch_lines(orc):
    """With g = 0.1 as a float (0.100000001...), 60 g overshoots 6 m: the
    last column still lies on the goal line, where a point's lines to the
    posts run along the defence area's back edge and enter it at its
    corner, (6, +-1.2)."""
    batch = synth.run_states(15, 1)
    batch["opp_pos"][0, 0] = (6.0, 1.2)      # a guard at rest on the corner
    batch["opp_vel"][0, 0] = (0.0, 0.0)
    batch["opp_pos"][0, 1] = (-6.0, 0.0)     # the second: out of the area
    prm = synth.run_oracle_params()
    r = orc.run_search(batch, prm, dense=True)
    st = oracle.dstate_of(batch, 0)
    top = orc.run_point(st, prm, (6.0, 4.5))
    assert r["score"][0, -1, -1] == top["score"]
    # both lines run down the goal line and enter at the corner, where the
    # guard stands: no time to either P or Q
    assert top["guard"] < 1e-6
    # one step in from the goal line the lines enter through the side
    # y = 1.2 left of the corner, and the guard needs time
    assert orc.run_point(st, prm, (5.9, 4.5))["guard"] > 1e-2


def check_edges_take_a_tolerance_of_g_over_1024(orc):
    """A point within g / 1024 (about 1e-4 m at 0.1 m) of the defence
    area's edge or of a zone cut counts as on it, so grid points on those
    lines do not depend on the rounding of i g."""
    st = _st()
    assert orc.run_point(st, PRM, (4.8 + 5e-5, 0.0))["candidate"]
    assert not orc.run_point(st, PRM, (4.8 + 2e-4, 0.0))["candidate"]
    assert orc.run_point(st, PRM, (5.5, 1.2 - 5e-5))["candidate"]
    assert not orc.run_point(st, PRM, (5.5, 1.2 - 2e-4))["candidate"]
    assert orc.run_zone(st, (3.0 - 5e-5, 1.0), PRM) == 3
    assert orc.run_zone(st, (3.0 - 2e-4, 1.0), PRM) == 1
    assert orc.run_zone(st, (1.0, -5e-5), PRM) == 1
    assert orc.run_zone(st, (1.0, -2e-4), PRM) == 0
    # on the float grid, column 48 (48 g = 4.80000007 with g the float
    # nearest 0.1) is on the area's front edge: a candidate at y = 0
    batch = synth.run_states(16, 1)
    r = orc.run_search(batch, synth.run_oracle_params(), dense=True)
    assert np.isfinite(r["score"][0, 45, 48])
    assert np.isinf(r["score"][0, 45, 49])


def check_zone_choice_hand_cases(orc):
    idx = [10, 20, 30, 40]
    sc = [0.5, 0.9, 1.0, 1.2]
    assert list(orc.run_choose(idx, sc, -1, 4)) == [3, 2, 1, 0]
    assert list(orc.run_choose(idx, sc, -1, 2)) == [3, 2, -1, -1]
    assert list(orc.run_choose(idx, sc, 3, 2)) == [2, 1, -1, -1]
    assert list(orc.run_choose(idx, sc, 2, 4)) == [3, 1, 0, -1]
    assert list(orc.run_choose(idx, sc, -1, 0)) == [-1] * 4
    # a zone without a point is skipped; ties go to the lower zone
    assert list(orc.run_choose([10, 20, -1, 40], [1, 1, -np.inf, 2], -1,
                                  3)) == [3, 0, 1, -1]
    assert list(orc.run_choose(idx, [0.5, 0.5, 1.0, 1.0], -1, 4)) == \
        [2, 3, 0, 1]


def check_pass_point_zone_is_avoided(orc):
    batch = synth.run_states(12, 4)
    prm = synth.run_oracle_params()
    pts = np.array([[5.0, 3.0], [1.0, -3.0], [-2.0, 0.0], [np.nan, np.nan]])
    r = orc.run_search(batch, prm, pass_points=pts)
    for s in range(4):
        av = orc.run_zone(oracle.dstate_of(batch, s), pts[s]) \
            if np.isfinite(pts[s]).all() else -1
        assert r["avoided"][s] == av
        assert av not in list(r["chosen"][s])
        assert list(r["chosen"][s]) == list(orc.run_choose(
            r["best_idx"][s], r["best_score"][s], av, 4))
    assert r["avoided"][2] == -1            # a pass into our own half


def check_mirror_symmetry(orc):
    """Mirroring the state in y mirrors the score grid (up to the rounding
    of the grid's y coordinates near the area's and the zones' edges)."""
    batch = synth.run_states(13, 3)
    prm = dict(synth.run_oracle_params(), spacing=0.125)  # exact in binary
    m = {k: (v.copy() if isinstance(v, np.ndarray) else v)
         for k, v in batch.items()}
    m["ball"][:, 1] *= -1
    m["opp_pos"][:, :, 1] *= -1
    m["opp_vel"][:, :, 1] *= -1
    a = orc.run_search(batch, prm, dense=True)["score"]
    b = orc.run_search(m, prm, dense=True)["score"][:, ::-1, :]
    both = np.isfinite(a) & np.isfinite(b)
    assert np.array_equal(np.isfinite(a), np.isfinite(b))
    assert np.allclose(a[both], b[both], rtol=0, atol=1e-12)


CHECKS = [
    check_zones_split_at_quarter_length_and_the_ball,
    check_distance_criteria_and_the_defence_area,
    check_angle_credit_is_a_band_off_the_goal_axis,
    check_guard_time_to_p_and_q_against_a_walk_along_the_lines,
    check_guards_are_only_the_opponents_inside_the_area,
    check_avoid_is_set_when_an_opponent_is_nearer_the_ball,
    check_score_is_the_weighted_sum_with_costs_signed,
    check_best_per_zone_is_the_argmax_of_the_dense_scores,
    check_ties_go_to_the_lowest_index,
    check_raster_ends_on_the_goal_and_touch_lines,
    check_edges_take_a_tolerance_of_g_over_1024,
    check_zone_choice_hand_cases,
    check_pass_point_zone_is_avoided,
    check_mirror_symmetry,
]


@pytest.mark.parametrize("chk", CHECKS, ids=[c.__name__[6:] for c in CHECKS])
def test_pin(chk):
    chk(oracle.default())
