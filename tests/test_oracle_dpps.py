"""Pins of the oracle's direction x power search (the paper's own
parameterisation of the passing-point search, Sec. 4.2; features of
Sec. 4.3).

The path rule against closed forms, the sampled first interception against
brute-force time stepping, a receiver on the pass line against the 1-D
closed forms written out here, the score of a hand case, and invariants
(more opponents, fewer teammates, mirror symmetry).
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


def test_path_is_the_stop_or_the_field_edge():
    st = _st()
    # 3 m/s at 0.5 m/s^2 stops after 9 m; the edge is 6 m away along +x
    assert oracle.dpps_path(st, (1.0, 0.0), 3.0) == (6.0, False)
    # 1 m/s stops after 1 m, well inside
    S, stopped = oracle.dpps_path(st, (0.0, 1.0), 1.0)
    assert stopped and math.isclose(S, 1.0, rel_tol=1e-15)
    # from (5, 4) along the diagonal the side line (y = 4.5) comes first
    c = math.sqrt(0.5)
    S, stopped = oracle.dpps_path(_st(ball=(5.0, 4.0)), (c, c), 6.5)
    assert not stopped and math.isclose(S, 0.5 / c, rel_tol=1e-12)


def _bang_bang_from_rest(d, vmax=3.25, amax=3.0):
    if d <= vmax * vmax / (2 * amax):
        return math.sqrt(2 * d / amax)
    return d / vmax + vmax / (2 * amax)


def test_receiver_on_the_line_matches_closed_forms():
    """A teammate standing on the pass line: the first sample it can reach
    no later than the ball, from the 1-D ball and bang-bang formulas."""
    for x0, v in ((2.0, 3.0), (0.7, 4.5), (5.5, 2.0), (1.0, 1.0)):
        st = _st(team=[(x0, 0.0, 0.0, 0.0)])
        S, stopped = oracle.dpps_path(st, (1.0, 0.0), v)
        want = math.inf
        for k in range(1, 65):
            s = k / 64 * S
            tb = v / 0.5 if (stopped and k == 64) else \
                (v - math.sqrt(v * v - 2 * 0.5 * s)) / 0.5
            T = _bang_bang_from_rest(abs(x0 - s))
            if T <= tb or (stopped and k == 64):
                want = max(T, tb)
                break
        t, k, who = oracle.dpps_group(st, st.team, (1.0, 0.0), v)
        if math.isinf(want):  # the ball outruns it to the field edge
            assert math.isinf(t) and who == -1 and k == 0
        else:
            assert who == 0 and math.isclose(t, want, rel_tol=1e-12), (x0, v)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sampled_interception_brackets_brute_force(seed):
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
        t, k, _ = oracle.dpps_group(st, st.team, u, v)
        S, stopped = oracle.dpps_path(st, u, v)
        # continuous first time any robot reaches the ball
        a, tc = 0.5, math.inf
        t_end = v / a if stopped else 2 * S / (v + math.sqrt(v * v - 2 * a * S))
        for tt in np.arange(0.0, t_end + 1e-4, 1e-4):
            s = min(v * tt - 0.5 * a * tt * tt, S)
            p = (s * u[0], s * u[1])
            T = min(oracle.intercept_time(r[:2], r[2:], p, 3.25, 3.0)
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


def test_score_of_a_hand_case():
    """A still receiver on the x axis, no opponents: the score is the
    receive time, the whole goal mouth, the goal distance, no refraction
    and the capped delta-time."""
    st = _st(team=[(2.0, 0.0, 0.0, 0.0)])
    c = oracle.dpps_candidate(st, PRM, 128, 64, 0, 30)
    assert c["feasible"] == 1.0 and c["receiver"] == 0.0
    v = 5 / 7 * (1.0 + 30 * 5.5 / 63)
    t, k, _ = oracle.dpps_group(st, st.team, (1.0, 0.0), v)
    S, _ = oracle.dpps_path(st, (1.0, 0.0), v)
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


def test_invariants_more_opponents_fewer_teammates_mirror():
    b = _batch(7)
    base = oracle.dpps_search(b, 32, 8, PRM, dense=True)
    # one more opponent: t_opp never rises, nothing becomes feasible
    b2 = dict(b)
    b2["opp_pos"] = np.concatenate([b["opp_pos"], [[[0.5, 0.5]]] * 3], 1)
    b2["opp_vel"] = np.concatenate([b["opp_vel"], [[[0.0, 0.0]]] * 3], 1)
    b2["n_opp"] = b["n_opp"] + 1
    more = oracle.dpps_search(b2, 32, 8, PRM, dense=True)
    assert np.all(more["t_opp"] <= base["t_opp"])
    assert np.all(more["feasible"] <= base["feasible"])
    # one teammate fewer: t_team never drops
    b3 = dict(b)
    b3["team_pos"], b3["team_vel"] = b["team_pos"][:, 1:], b["team_vel"][:, 1:]
    fewer = oracle.dpps_search(b3, 32, 8, PRM, dense=True)
    assert np.all(fewer["t_team"] >= base["t_team"])
    # mirror y -> -y: direction i maps to (32 - i) mod 32
    bm = dict(b)
    for k in ("ball", "team_pos", "team_vel", "opp_pos", "opp_vel"):
        bm[k] = b[k] * np.array([1.0, -1.0])
    mir = oracle.dpps_search(bm, 32, 8, PRM, dense=True)
    perm = np.array([((32 - i) % 32) * 8 + j for i in range(32)
                     for j in range(8)])
    assert np.allclose(mir["t_team"][:, perm], base["t_team"], rtol=1e-9)
    assert np.allclose(mir["t_opp"][:, perm], base["t_opp"], rtol=1e-9)


def test_search_best_is_the_dense_argmax_and_empty_teams_fail():
    b = _batch(8)
    r = oracle.dpps_search(b, 32, 8, PRM, dense=True)
    for s in range(3):
        sc = np.where(r["feasible"][s] == 1, r["score"][s], -np.inf)
        if r["best_idx"][s] >= 0:
            assert r["best_idx"][s] == int(np.argmax(sc))
            assert r["best_score"][s] == sc.max()
        assert r["n_feasible"][s] == int(r["feasible"][s].sum())
    b["team_pos"], b["team_vel"] = b["team_pos"][:, :0], b["team_vel"][:, :0]
    r = oracle.dpps_search(b, 32, 8, PRM)
    assert np.all(r["best_idx"] == -1) and np.all(r["n_feasible"] == 0)


def test_pass_power_inverts_the_ball_model():
    """Eq. 1-2: the rolling speed covers the distance in the receiver's
    arrival time plus the buffer (d = v1 t - a t^2 / 2), the kick power is
    7/5 of it, limited to the robot's range."""
    st = _st(team=[(3.0, 1.0, 0.0, 0.0)])
    r = oracle.pass_power(st, 0, (3.0, 0.0), buffer=0.3)
    T = math.sqrt(2 * 1.0 / 3.0)            # from rest, 1 m
    assert math.isclose(r["t_recv"], T, rel_tol=1e-12)
    t = T + 0.3
    assert math.isclose(r["t_pass"], t, rel_tol=1e-12)
    assert math.isclose(3.0, r["v1"] * t - 0.25 * t * t, rel_tol=1e-12)
    assert math.isclose(r["v0"], r["v1"] * 7 / 5, rel_tol=1e-12)
    assert r["clamped"] == 0.0
    # a late receiver close by: the slowest ball that still gets there
    slow = oracle.pass_power(_st(team=[(0.5, 4.0, 0.0, 0.0)]), 0, (0.5, 0.0))
    assert math.isclose(slow["v1"], math.sqrt(2 * 0.5 * 0.5), rel_tol=1e-12)
    # a far target reached early: more than the robot can kick
    far = oracle.pass_power(_st(team=[(5.9, 0.0, 0.0, 0.0)]), 0, (6.0, 0.0),
                            buffer=0.0)
    assert far["clamped"] == 1.0 and far["v0"] == 6.5


def test_shooting_decision():
    """Sec. 4.4: the open angle and its middle direction, the ball's time
    to the goal line, and the opponents along the shot."""
    c = (3.0, 0.5)
    st = _st()
    r = oracle.shoot(st, c, theta_min=0.1)
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
    blocked = oracle.shoot(side, c, v_shot=3.0, theta_min=0.0)
    assert math.isclose(blocked["theta"], hi - lo, rel_tol=1e-12)
    assert blocked["t_opp"] < blocked["t_line"] and blocked["shoot"] == 0.0
    assert oracle.shoot(side, c, v_shot=6.5, theta_min=0.0)["shoot"] == 1.0
    # too narrow an angle, or a ball that stops short: no shot
    assert oracle.shoot(st, c, theta_min=1.0)["shoot"] == 0.0
    weak = oracle.shoot(st, c, v_shot=1.0)
    assert math.isinf(weak["t_line"]) and weak["shoot"] == 0.0
