"""Pins of the oracle's direction x power search (the paper's own
parameterisation of the passing-point search, Sec. 4.2; features of
Sec. 4.3).

The path rule against closed forms, the sampled first interception against
brute-force time stepping, a receiver on the pass line against the 1-D
closed forms written out here, the score of a hand case, and invariants
(more opponents, fewer teammates, mirror symmetry).  Each check takes an
oracle build, so the mutant tests can run them against copies with planted
mistakes.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle

SC = {"ball_x": 0.0, "ball_y": 0.0, "ball_decel": 0.5, "vmax": 3.25,
      "amax": 3.0, "field_len": 12.0, "field_wid": 9.0, "goal_width": 1.8}
PRM = dict(vlo=1.0, vhi=6.5, slide=5 / 7, tau_delta=0.0, delta_cap=1.0,
           w_time=1.0, w_angle=1.0, w_dist=1.0, w_refr=1.0, w_delta=1.0,
           robot_radius=0.09, reach_radius=0.0, min_time=0.0)


def _st(team=(), opp=(), ball=(0.0, 0.0), K=64):
    sc = dict(SC, ball_x=ball[0], ball_y=ball[1])
    return oracle.DState(sc, np.array(team, float).reshape(-1, 4),
                         np.array(opp, float).reshape(-1, 4), K)


def check_path_is_the_stop_or_the_field_edge(orc):
    st = _st()
    # 3 m/s at 0.5 m/s^2 stops after 9 m; the edge is 6 m away along +x
    assert orc.dpps_path(st, (1.0, 0.0), 3.0) == (6.0, False)
    # 1 m/s stops after 1 m, well inside
    S, stopped = orc.dpps_path(st, (0.0, 1.0), 1.0)
    assert stopped and math.isclose(S, 1.0, rel_tol=1e-15)
    # from (5, 4) along the diagonal the side line (y = 4.5) comes first
    c = math.sqrt(0.5)
    S, stopped = orc.dpps_path(_st(ball=(5.0, 4.0)), (c, c), 6.5)
    assert not stopped and math.isclose(S, 0.5 / c, rel_tol=1e-12)


def _bang_bang_from_rest(d, vmax=3.25, amax=3.0):
    if d <= vmax * vmax / (2 * amax):
        return math.sqrt(2 * d / amax)
    return d / vmax + vmax / (2 * amax)


def check_receiver_on_the_line_matches_closed_forms(orc):
    """A teammate standing on the pass line: the first sample it can reach
    no later than the ball, from the 1-D ball and bang-bang formulas."""
    for x0, v in ((2.0, 3.0), (0.7, 4.5), (5.5, 2.0), (1.0, 1.0)):
        st = _st(team=[(x0, 0.0, 0.0, 0.0)])
        S, stopped = orc.dpps_path(st, (1.0, 0.0), v)
        want, want_k = math.inf, 0
        for k in range(1, 65):
            s = k / 64 * S
            tb = v / 0.5 if (stopped and k == 64) else \
                (v - math.sqrt(v * v - 2 * 0.5 * s)) / 0.5
            T = _bang_bang_from_rest(abs(x0 - s))
            if T <= tb or (stopped and k == 64):
                want, want_k = max(T, tb), k
                break
        t, k, who = orc.dpps_group(st, st.team, (1.0, 0.0), v)
        if math.isinf(want):  # the ball outruns it to the field edge
            assert math.isinf(t) and who == -1 and k == 0
        else:
            assert who == 0 and math.isclose(t, want, rel_tol=1e-12), (x0, v)
            assert k == want_k, (x0, v, k, want_k)


def check_sampled_interception_brackets_brute_force(orc, seed=1):
    """The sampled first interception is never earlier than the continuous
    one (found by 0.1 ms time stepping) and at most one sample later."""
    rng = np.random.default_rng(seed)
    for _ in range(6):
        n = 4
        robots = np.concatenate([rng.uniform(-4, 4, (n, 2)),
                                 rng.uniform(-2, 2, (n, 2))], axis=1)
        st = _st(team=robots)
        phi = rng.uniform(0, 2 * math.pi)
        u = (math.cos(phi), math.sin(phi))
        v = rng.uniform(1.0, 4.6)
        t, k, _ = orc.dpps_group(st, st.team, u, v)
        S, stopped = orc.dpps_path(st, u, v)
        # continuous first time any robot reaches the ball
        a, tc = 0.5, math.inf
        t_end = v / a if stopped else 2 * S / (v + math.sqrt(v * v - 2 * a * S))
        for tt in np.arange(0.0, t_end + 1e-4, 1e-4):
            s = min(v * tt - 0.5 * a * tt * tt, S)
            p = (s * u[0], s * u[1])
            T = min(orc.intercept_time(r[:2], r[2:], p, 3.25, 3.0)
                    for r in robots)
            if T <= tt:
                tc = tt
                break
        if not math.isfinite(t):
            assert not math.isfinite(tc) or (stopped is False)
            continue
        if stopped and k == 64 and not math.isfinite(tc):
            continue  # only the ball at rest is reached
        dt = t_end / 64 * 4  # a sample step in time is at most this long
        assert tc - 2e-4 <= t <= tc + dt, (t, tc)


def check_stop_sample_rule(orc):
    """A ball that stops (1 m/s at 0.5 m/s^2: 1 m in 2 s) is taken at rest
    at its last sample by whoever comes: a receiver 4.3 m off the rest
    point arrives at 1.865 s and gets it at the stop time 2 s; one 5 m off
    arrives after it stopped, at 2.080 s (bang-bang from rest, written out
    here); neither reaches an earlier sample in time."""
    for ry, want in ((0.3, 2.0), (1.0, 5.0 / 3.25 + 3.25 / 6.0)):
        st = _st(team=[(1.0, ry, 0.0, 0.0)], ball=(0.0, -4.0))
        S, stopped = orc.dpps_path(st, (1.0, 0.0), 1.0)
        assert stopped and math.isclose(S, 1.0, rel_tol=1e-15)
        t, k, who = orc.dpps_group(st, st.team, (1.0, 0.0), 1.0)
        assert k == 64 and who == 0, (ry, k)
        assert math.isclose(t, want, rel_tol=1e-12), (ry, t, want)


def check_refraction_of_a_hand_case(orc):
    """A pass straight up the field (direction 32 of 128) to a still
    receiver on that line, no opponents: the refraction term is the turn
    from the pass direction (0, 1) to the shot at the goal centre from the
    receive point, acos(-ry / |goal - r|); the rest as in the hand case
    along x."""
    st = _st(team=[(0.0, 2.0, 0.0, 0.0)])
    prm = dict(PRM, slide=1.0)
    c = orc.dpps_candidate(st, prm, 128, 64, 32, 20)
    assert c["feasible"] == 1.0 and c["receiver"] == 0.0
    v = 1.0 + 20 * 5.5 / 63
    u = (math.cos(math.pi / 2), math.sin(math.pi / 2))
    t, k, _ = orc.dpps_group(st, st.team, u, v)
    S, _ = orc.dpps_path(st, u, v)
    ry = k / 64 * S * u[1]
    rx = k / 64 * S * u[0]
    gx, gy = 6.0 - rx, -ry
    dg = math.hypot(gx, gy)
    theta = math.atan2(0.9 - ry, gx) - math.atan2(-0.9 - ry, gx)
    refr = math.acos((u[0] * gx + u[1] * gy) / dg)
    assert refr > 1.7
    want = -t + theta / math.pi - dg / 15.0 - refr / math.pi + 1.0
    assert math.isclose(c["score"], want, rel_tol=1e-12), (c, want)
    # the same pass with the refraction weight doubled loses refr / pi
    c2 = orc.dpps_candidate(st, dict(prm, w_refr=2.0), 128, 64, 32, 20)
    assert math.isclose(c2["score"], want - refr / math.pi, rel_tol=1e-12)


def check_score_of_a_hand_case(orc):
    """A still receiver on the x axis, no opponents: the score is the
    receive time, the whole goal mouth, the goal distance, no refraction
    and the capped delta-time."""
    st = _st(team=[(2.0, 0.0, 0.0, 0.0)])
    c = orc.dpps_candidate(st, PRM, 128, 64, 0, 30)
    assert c["feasible"] == 1.0 and c["receiver"] == 0.0
    v = 5 / 7 * (1.0 + 30 * 5.5 / 63)
    t, k, _ = orc.dpps_group(st, st.team, (1.0, 0.0), v)
    S, _ = orc.dpps_path(st, (1.0, 0.0), v)
    px = k / 64 * S
    theta = math.atan2(0.9, 6 - px) - math.atan2(-0.9, 6 - px)
    want = -t + theta / math.pi - (6 - px) / 15.0 - 0.0 + 1.0
    assert math.isclose(c["score"], want, rel_tol=1e-12)
    assert c["rx"] == px and c["ry"] == 0.0


def _batch(seed, S=3, nt=5, no=5):
    rng = np.random.default_rng(seed)
    b = {"ball": rng.uniform([-5, -4], [5, 4], (S, 2)),
         "team_pos": rng.uniform([-6, -4.5], [6, 4.5], (S, nt, 2)),
         "team_vel": rng.uniform(-2, 2, (S, nt, 2)),
         "opp_pos": rng.uniform([-6, -4.5], [6, 4.5], (S, no, 2)),
         "opp_vel": rng.uniform(-2, 2, (S, no, 2)),
         "n_opp": np.full(S, no), "K": np.full(S, 32)}
    for k in ("ball_decel", "vmax", "amax", "field_len", "field_wid",
              "goal_width"):
        b[k] = np.full(S, SC[k])
    return b


def check_invariants_more_opponents_fewer_teammates_mirror(orc):
    b = _batch(7)
    base = orc.dpps_search(b, 32, 8, PRM, dense=True)
    # one more opponent: t_opp never rises, nothing becomes feasible
    b2 = dict(b)
    b2["opp_pos"] = np.concatenate([b["opp_pos"], [[[0.5, 0.5]]] * 3], 1)
    b2["opp_vel"] = np.concatenate([b["opp_vel"], [[[0.0, 0.0]]] * 3], 1)
    b2["n_opp"] = b["n_opp"] + 1
    more = orc.dpps_search(b2, 32, 8, PRM, dense=True)
    assert np.all(more["t_opp"] <= base["t_opp"])
    assert np.all(more["feasible"] <= base["feasible"])
    # one teammate fewer: t_team never drops
    b3 = dict(b)
    b3["team_pos"], b3["team_vel"] = b["team_pos"][:, 1:], b["team_vel"][:, 1:]
    fewer = orc.dpps_search(b3, 32, 8, PRM, dense=True)
    assert np.all(fewer["t_team"] >= base["t_team"])
    # mirror y -> -y: direction i maps to (32 - i) mod 32
    bm = dict(b)
    for k in ("ball", "team_pos", "team_vel", "opp_pos", "opp_vel"):
        bm[k] = b[k] * np.array([1.0, -1.0])
    mir = orc.dpps_search(bm, 32, 8, PRM, dense=True)
    perm = np.array([((32 - i) % 32) * 8 + j for i in range(32)
                     for j in range(8)])
    assert np.allclose(mir["t_team"][:, perm], base["t_team"], rtol=1e-9)
    assert np.allclose(mir["t_opp"][:, perm], base["t_opp"], rtol=1e-9)


def check_search_best_is_the_dense_argmax_and_empty_teams_fail(orc):
    b = _batch(8)
    r = orc.dpps_search(b, 32, 8, PRM, dense=True)
    for s in range(3):
        sc = np.where(r["feasible"][s] == 1, r["score"][s], -np.inf)
        if r["best_idx"][s] >= 0:
            assert r["best_idx"][s] == int(np.argmax(sc))
            assert r["best_score"][s] == sc.max()
        assert r["n_feasible"][s] == int(r["feasible"][s].sum())
    b["team_pos"], b["team_vel"] = b["team_pos"][:, :0], b["team_vel"][:, :0]
    r = orc.dpps_search(b, 32, 8, PRM)
    assert np.all(r["best_idx"] == -1) and np.all(r["n_feasible"] == 0)


def check_pass_power_inverts_the_ball_model(orc):
    """Eq. 1-2: the rolling speed covers the distance in the receiver's
    arrival time plus the buffer (d = v1 t - a t^2 / 2), the kick power is
    7/5 of it, limited to the robot's range."""
    st = _st(team=[(3.0, 1.0, 0.0, 0.0)])
    r = orc.pass_power(st, 0, (3.0, 0.0), buffer=0.3)
    T = math.sqrt(2 * 1.0 / 3.0)            # from rest, 1 m
    assert math.isclose(r["t_recv"], T, rel_tol=1e-12)
    t = T + 0.3
    assert math.isclose(r["t_pass"], t, rel_tol=1e-12)
    assert math.isclose(3.0, r["v1"] * t - 0.25 * t * t, rel_tol=1e-12)
    assert math.isclose(r["v0"], r["v1"] * 7 / 5, rel_tol=1e-12)
    assert r["clamped"] == 0.0
    # a late receiver close by: the slowest ball that still gets there
    slow = orc.pass_power(_st(team=[(0.5, 4.0, 0.0, 0.0)]), 0, (0.5, 0.0))
    assert math.isclose(slow["v1"], math.sqrt(2 * 0.5 * 0.5), rel_tol=1e-12)
    # a far target reached early: more than the robot can kick
    far = orc.pass_power(_st(team=[(5.9, 0.0, 0.0, 0.0)]), 0, (6.0, 0.0),
                            buffer=0.0)
    assert far["clamped"] == 1.0 and far["v0"] == 6.5


def check_shooting_decision(orc):
    """Sec. 4.4: the open angle and its middle direction, the ball's time
    to the goal line, and the opponents along the shot."""
    c = (3.0, 0.5)
    st = _st()
    r = orc.shoot(st, c, theta_min=0.1)
    lo, hi = math.atan2(-0.9 - 0.5, 3.0), math.atan2(0.9 - 0.5, 3.0)
    assert math.isclose(r["theta"], hi - lo, rel_tol=1e-12)
    assert math.isclose(r["dir"], 0.5 * (lo + hi), rel_tol=1e-12)
    v = 6.5 * 5 / 7
    s = 3.0 / math.cos(r["dir"])
    assert math.isclose(r["t_line"], (v - math.sqrt(v * v - s)) / 0.5,
                        rel_tol=1e-9)
    assert r["shoot"] == 1.0 and math.isinf(r["t_opp"])
    # an opponent running in from the side (outside the mouth's angle)
    # takes a slower shot first
    side = _st(opp=[(4.5, 2.5, 0.0, -3.0)])
    blocked = orc.shoot(side, c, v_shot=3.0, theta_min=0.0)
    assert math.isclose(blocked["theta"], hi - lo, rel_tol=1e-12)
    assert blocked["t_opp"] < blocked["t_line"] and blocked["shoot"] == 0.0
    assert orc.shoot(side, c, v_shot=6.5, theta_min=0.0)["shoot"] == 1.0
    # too narrow an angle, or a ball that stops short: no shot
    assert orc.shoot(st, c, theta_min=1.0)["shoot"] == 0.0
    weak = orc.shoot(st, c, v_shot=1.0)
    assert math.isinf(weak["t_line"]) and weak["shoot"] == 0.0


CHECKS = [
    check_path_is_the_stop_or_the_field_edge,
    check_receiver_on_the_line_matches_closed_forms,
    check_sampled_interception_brackets_brute_force,
    check_score_of_a_hand_case,
    check_stop_sample_rule,
    check_refraction_of_a_hand_case,
    check_invariants_more_opponents_fewer_teammates_mirror,
    check_search_best_is_the_dense_argmax_and_empty_teams_fail,
    check_pass_power_inverts_the_ball_model,
    check_shooting_decision,
]


@pytest.mark.parametrize("chk", CHECKS, ids=[c.__name__[6:] for c in CHECKS])
def test_pin(chk):
    chk(oracle.default())


@pytest.mark.parametrize("seed", [2, 3])
def test_sampled_interception_more_seeds(seed):
    check_sampled_interception_brackets_brute_force(oracle.default(), seed)
