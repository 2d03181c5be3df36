"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper and the mathematics fix:
hand-derived special cases (tests/golden/hand_cases.json), brute-force time
stepping (tests/brute.py), ray casting, and invariants of the definition.
The pins are chosen so that a plausible slip in the oracle (a dropped term,
a sign, an index, a swapped operand) fails at least one of them; the
mutation tests in test_oracle_mutants.py plant such slips and check that.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import brute
from paper_1909_07717_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
HAND = json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))
PARAMS = synth.DEFAULT_PARAMS


def _orc(o=None):
    return o if o is not None else oracle.default()


def _state(ball=(0.0, 0.0), opps=(), decel=0.5, vmax=3.25, amax=3.0, L=12.0,
           W=9.0, gw=1.8, K=8):
    opp = np.array([list(p) + list(u) for p, u in opps], float).reshape(-1, 4)
    sc = dict(ball_x=ball[0], ball_y=ball[1], ball_decel=decel, vmax=vmax,
              amax=amax, field_len=L, field_wid=W, goal_width=gw)
    return oracle.State(sc, opp, K)


def _exp(x):
    return math.inf if x == "inf" else float(x)


# ---------------------------------------------------------------- hand cases
def check_hand_ball(o=None):
    for c in HAND["ball_time"]:
        got = _orc(o).ball_time(c["s"], c["v"], c["a"])
        exp = _exp(c["expect"])
        assert (got == exp) if math.isinf(exp) else got == pytest.approx(
            exp, abs=1e-12), c["why"]


def check_hand_intercept(o=None):
    for c in HAND["intercept_time"]:
        got = _orc(o).intercept_time(c["o"], c["u"], c["p"], c["vmax"],
                                     c["amax"], c["reach"])
        assert got == pytest.approx(c["expect"], abs=1e-12), c["why"]


def check_hand_shot(o=None):
    for c in HAND["shot_angle"]:
        st = _state(opps=[(p, (0, 0)) for p in c["opps"]], L=c["L"],
                    gw=c["gw"])
        got = _orc(o).shot_angle(st, c["c"], c["r"])
        assert got == pytest.approx(c["expect"], abs=1e-12), c["why"]


def check_hand_score(o=None):
    for c in HAND["score"]:
        st = _state(ball=c["ball"], L=c["L"], W=c["W"], gw=c["gw"],
                    decel=c["decel"], K=c["K"])
        m, reach, _ = _orc(o).margin(st, c["c"], c["v"])
        assert reach and m == math.inf
        got = _orc(o).score(st, PARAMS, c["c"], m)
        assert got == pytest.approx(c["expect"], abs=1e-12), c["why"]


def check_hand_grid(o=None):
    for c in HAND["grid"]:
        nx, ny, x0, y0 = _orc(o).grid(c["L"], c["W"], np.float32(c["g"]))
        assert (nx, ny) == (c["nx"], c["ny"]), c["why"]
        assert (x0, y0) == (-c["L"] / 2, -c["W"] / 2)


def test_hand_ball():
    check_hand_ball()


def test_hand_intercept():
    check_hand_intercept()


def test_hand_shot():
    check_hand_shot()


def test_hand_score():
    check_hand_score()


def test_hand_grid():
    check_hand_grid()


# ------------------------------------------------------ brute-force stepping
def check_ball_vs_sim(o=None, n=400, seed=11):
    """Closed form against a 1 ms time-stepped rolling ball (Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(1.0, 6.5, n)
    a = rng.uniform(0.3, 0.7, n)
    stop = v * v / (2 * a)
    s = rng.uniform(0.0, 1.3, n) * np.minimum(stop, 15.0)
    sim = brute.ball_arrival_sim(s, v, a)
    got = np.array([_orc(o).ball_time(*x) for x in zip(s, v, a)])
    clear = np.abs(s - stop) > 0.02 * stop  # the last step rounds the stop
    both_inf = np.isinf(got) & np.isinf(sim)
    fin = np.isfinite(got) & np.isfinite(sim)
    assert np.all((both_inf | fin)[clear])
    sel = fin & clear
    assert np.all(np.abs(got[sel] - sim[sel]) <= 1.0001e-3)
    # The kinematic identity s = v t - a t^2 / 2 holds at the returned time.
    f = np.isfinite(got)
    assert np.allclose(v[f] * got[f] - 0.5 * a[f] * got[f] ** 2, s[f],
                       atol=1e-9)


def check_intercept_vs_sim(o=None, n=300, seed=12):
    """Closed form against a 1 ms time-stepped robot (Sec. 4.2 reading)."""
    rng = np.random.default_rng(seed)
    for i in range(n):
        op = rng.uniform(-6, 6, 2)
        p = op + rng.uniform(-4, 4, 2) * rng.choice([0.02, 0.3, 1.0])
        sp = rng.uniform(0, 4.0)  # sometimes faster than vmax: clamped
        hd = rng.uniform(0, 2 * math.pi)
        u = sp * np.array([math.cos(hd), math.sin(hd)])
        vmax = rng.uniform(2.0, 4.0)
        amax = rng.uniform(1.5, 4.0)
        reach = rng.choice([0.0, 0.09])
        got = _orc(o).intercept_time(op, u, p, vmax, amax, reach)
        sim = brute.robot_arrival_sim(op, u, p, vmax, amax, reach)
        assert abs(got - sim) <= 1.0001e-3, (op, u, p, vmax, amax, reach,
                                               got, sim)


def check_margin_vs_sim(o=None, seed=13):
    """Whole candidates: every robot and the ball stepped to every sample."""
    rng = np.random.default_rng(seed)
    checked = 0
    for trial in range(12):
        ball = rng.uniform([-6, -4.5], [6, 4.5])
        opps = []
        for j in range(rng.integers(1, 4)):
            hd = rng.uniform(0, 2 * math.pi)
            sp = rng.uniform(0, 3.25)
            opps.append((rng.uniform([-6, -4.5], [6, 4.5]),
                         sp * np.array([math.cos(hd), math.sin(hd)])))
        K = int(rng.choice([3, 4, 6]))
        st = _state(ball=ball, opps=opps, K=K)
        c = ball + rng.uniform(-5, 5, 2)
        v = float(rng.choice([2.0, 4.0, 6.5]))
        reach = float(rng.choice([0.0, 0.09]))
        m, reachable, T = _orc(o).margin(st, c, v, reach)
        ms, Ts, tbs = brute.candidate_margin_sim(ball, opps, c, v, 0.5, 3.25,
                                                 3.0, K, reach)
        assert np.all(np.abs(np.array(Ts) - T) <= 1.0001e-3)
        if not reachable:
            assert m == -math.inf and math.isinf(tbs[-1])
            continue
        assert abs(m - ms) <= 2.0001e-3, (m, ms)
        checked += 1
    assert checked >= 4


def check_intercept_is_minimal(o=None, seed=14, n=40):
    """No admissible acceleration profile along the line arrives sooner."""
    rng = np.random.default_rng(seed)
    dt = 1e-3
    for _ in range(n):
        d = rng.uniform(0.05, 6.0)
        w = rng.uniform(-3.25, 3.25)
        vmax, amax = 3.25, 3.0
        t_star = _orc(o).intercept_time((0, 0), (w, 0), (d, 0), vmax, amax)
        for _ in range(5):
            x, vel, t = 0.0, w, 0.0
            acc = rng.uniform(-amax, amax, 20000)
            hit = math.inf
            for i in range(20000):
                vnew = min(max(vel + acc[i] * dt, -vmax), vmax)
                x += 0.5 * (vel + vnew) * dt
                vel = vnew
                t += dt
                if x >= d:
                    hit = t
                    break
                if t > t_star + 0.01:
                    break
            assert hit >= t_star - 1e-9


def test_ball_vs_sim():
    check_ball_vs_sim()


def test_intercept_vs_sim():
    check_intercept_vs_sim()


def test_margin_vs_sim():
    check_margin_vs_sim()


def test_intercept_is_minimal():
    check_intercept_is_minimal(n=10)


# --------------------------------------------------------------- invariants
def _random_state(rng, n_opp=5, K=16):
    opps = []
    for _ in range(n_opp):
        hd = rng.uniform(0, 2 * math.pi)
        opps.append((rng.uniform([-6, -4.5], [6, 4.5]),
                     rng.uniform(0, 3.25) * np.array([math.cos(hd),
                                                      math.sin(hd)])))
    ball = rng.uniform([-6, -4.5], [6, 4.5])
    return ball, opps, _state(ball=ball, opps=opps, K=K)


def check_invariants(o=None, seed=15):
    rng = np.random.default_rng(seed)
    orc = _orc(o)
    for trial in range(30):
        ball, opps, st = _random_state(rng, n_opp=int(rng.integers(1, 7)),
                                       K=int(rng.choice([8, 16, 32])))
        c = rng.uniform([-6, -4.5], [6, 4.5])
        v = float(rng.choice([2.0, 3.5, 5.0, 6.5]))
        m, reach, T = orc.margin(st, c, v)
        # (i) sample nesting: the midpoint receiver with K/2 samples sees
        # exactly the first K/2 samples of the full pass.
        mid = 0.5 * (ball + c)
        half = _state(ball=ball, opps=opps, K=st.K // 2)
        mh, rh, Th = orc.margin(half, mid, v)
        assert np.allclose(Th, T[: st.K // 2], rtol=0, atol=1e-9)
        if reach:
            assert rh and mh >= m - 1e-9
        # (ii) removing an opponent never lowers the margin.
        drop = int(rng.integers(0, len(opps)))
        fewer = _state(ball=ball, opps=opps[:drop] + opps[drop + 1:], K=st.K)
        mf, _, Tf = orc.margin(fewer, c, v)
        assert np.all(Tf >= T - 1e-12)
        assert mf >= m - 1e-12
        # (iii) opponent order does not matter.
        perm = [opps[i] for i in rng.permutation(len(opps))]
        mp, _, Tp = orc.margin(_state(ball=ball, opps=perm, K=st.K), c, v)
        assert np.array_equal(Tp, T) and (mp == m or (math.isnan(mp)
                                                      and math.isnan(m)))
        # (iv) mirroring y -> -y mirrors everything.
        mir = [((p[0], -p[1]), (u[0], -u[1])) for p, u in opps]
        mstate = _state(ball=(ball[0], -ball[1]), opps=mir, K=st.K)
        mm, _, Tm = orc.margin(mstate, (c[0], -c[1]), v)
        assert np.allclose(Tm, T, atol=1e-12)
        assert mm == pytest.approx(m, abs=1e-12) or mm == m
        sa = orc.shot_angle(st, c, 0.09)
        assert orc.shot_angle(mstate, (c[0], -c[1]), 0.09) == pytest.approx(
            sa, abs=1e-12)
        # (v) a faster kick never arrives later at any sample.
        if reach and v < 6.5:
            m2, r2, _ = orc.margin(st, c, 6.5)
            D = math.hypot(*(c - ball))
            for k in range(1, st.K + 1):
                s = k / st.K * D
                assert orc.ball_time(s, 6.5, 0.5) <= orc.ball_time(s, v, 0.5)


def check_intercept_monotone(o=None, seed=16):
    """Intercept time never grows with vmax, amax or speed toward the point."""
    rng = np.random.default_rng(seed)
    orc = _orc(o)
    for _ in range(300):
        d = rng.uniform(0.01, 8)
        vmax = rng.uniform(2, 4)
        amax = rng.uniform(1, 4)
        # |w| <= vmax: beyond it the clamp makes a larger vmax release more
        # receding speed, and the monotonicity in vmax no longer holds.
        w = rng.uniform(-vmax, vmax - 0.2)
        t = orc.intercept_time((0, 0), (w, 0), (d, 0), vmax, amax)
        assert orc.intercept_time((0, 0), (w, 0), (d, 0), vmax * 1.1,
                                  amax) <= t + 1e-12
        assert orc.intercept_time((0, 0), (w, 0), (d, 0), vmax,
                                  amax * 1.1) <= t + 1e-12
        assert orc.intercept_time((0, 0), (w + 0.2, 0), (d, 0), vmax,
                                  amax) <= t + 1e-12
        assert orc.intercept_time((0, 0), (w, 0), (d * 1.1, 0), vmax,
                                  amax) >= t - 1e-12
        # continuity across the accelerate / cruise switch
        dtop = (vmax ** 2 - w ** 2) / (2 * amax)
        lo = orc.intercept_time((0, 0), (w, 0), (dtop * (1 - 1e-9), 0), vmax,
                                amax)
        hi = orc.intercept_time((0, 0), (w, 0), (dtop * (1 + 1e-9), 0), vmax,
                                amax)
        assert abs(hi - lo) < 1e-6


def test_invariants():
    check_invariants()


def test_intercept_monotone():
    check_intercept_monotone()


# ----------------------------------------------------------------- geometry
def check_shot_vs_rays(o=None, seed=17, n=25):
    """Shot angle against a 10^5-ray sweep with exact disc intersection."""
    rng = np.random.default_rng(seed)
    orc = _orc(o)
    for trial in range(n):
        c = rng.uniform([-5.5, -4.0], [5.9, 4.0])
        k = int(rng.integers(0, 6))
        # bias opponents toward the shot cone so they actually block
        opp = []
        for _ in range(k):
            t = rng.uniform(0.1, 1.0)
            tgt = np.array([6.0, rng.uniform(-1.2, 1.2)])
            opp.append(c + t * (tgt - c) + rng.normal(0, 0.15, 2))
        st = _state(opps=[(p, (0, 0)) for p in opp])
        got = orc.shot_angle(st, c, 0.09)
        exp, step = brute.shot_angle_rays(c, opp, 12.0, 1.8, 0.09)
        assert abs(got - exp) <= 2 * step + 1e-9, (c, opp, got, exp)


def check_shot_closed_form(o=None, seed=18):
    """No opponents: the angle between the two post directions."""
    rng = np.random.default_rng(seed)
    st = _state()
    for _ in range(200):
        c = rng.uniform([-6, -4.5], [5.99, 4.5])
        A = np.array([6.0, -0.9]) - c
        B = np.array([6.0, 0.9]) - c
        exp = math.atan2(abs(A[0] * B[1] - A[1] * B[0]), A @ B)
        assert _orc(o).shot_angle(st, c, 0.09) == pytest.approx(exp,
                                                               abs=1e-12)


def check_score_closed_form(o=None, seed=19):
    """Score with no opponents (Eq. 3): angle/pi - dist/diag + capped margin."""
    rng = np.random.default_rng(seed)
    orc = _orc(o)
    for _ in range(100):
        c = rng.uniform([-6, -4.5], [5.99, 4.5])
        m = rng.uniform(-0.5, 2.0)
        w = dict(PARAMS)
        w.update(w_angle=rng.uniform(0, 2), w_dist=rng.uniform(0, 2),
                 w_margin=rng.uniform(0, 2), margin_cap=rng.uniform(0.2, 1.5))
        A = np.array([6.0, -0.9]) - c
        B = np.array([6.0, 0.9]) - c
        ang = math.atan2(abs(A[0] * B[1] - A[1] * B[0]), A @ B)
        exp = (w["w_angle"] * ang / math.pi
               - w["w_dist"] * math.hypot(6.0 - c[0], c[1]) / 15.0
               + w["w_margin"] * min(m, w["margin_cap"]))
        assert orc.score(_state(), w, c, m) == pytest.approx(exp, abs=1e-12)


def test_shot_vs_rays():
    check_shot_vs_rays()


def test_shot_closed_form():
    check_shot_closed_form()


def test_score_closed_form():
    check_score_closed_form()


# -------------------------------------------------------------- full search
def _grid(L, W, g, o=None):
    nx, ny, x0, y0 = _orc(o).grid(L, W, g)
    return (float(np.float32(g)), nx, ny, x0, y0)


def check_search_consistency(o=None):
    orc = _orc(o)
    b = synth.ssl_states(5, 3, K=8, n_opp=4)
    grid = _grid(12.0, 9.0, 0.5, o)
    speeds = [2.0, 4.5]
    out = orc.search(b, grid, speeds, PARAMS, dense=True, want_T=True)
    g, nx, ny, x0, y0 = grid
    P = nx * ny
    for s in range(3):
        st = oracle.state_of(b, s)
        feas = out["feasible"][s].reshape(-1).astype(bool)
        sc = out["score"][s].reshape(-1)
        assert out["n_feasible"][s] == feas.sum()
        if feas.any():
            best = np.max(sc[feas])
            first = int(np.flatnonzero(feas & (sc == best))[0])
            assert out["best_idx"][s] == first
            assert out["best_score"][s] == best
        else:
            assert out["best_idx"][s] == -1
        # spot-check candidates against the per-candidate entry points
        rng = np.random.default_rng(s)
        for idx in rng.integers(0, 2 * P, 12):
            v, p = divmod(int(idx), P)
            iy, ix = divmod(p, nx)
            c = (x0 + ix * g, y0 + iy * g)
            m, reach, T = orc.margin(st, c, speeds[v])
            assert out["margin"][s, v, p] == m
            if v == 0:
                assert np.array_equal(out["T"][s, p, : st.K], T)
            ok = reach and m > PARAMS["tau_safe"]
            assert bool(out["feasible"][s, v, p]) == ok


def check_search_tie_rule(o=None):
    """All feasible candidates score the same: the smallest index wins."""
    orc = _orc(o)
    b = synth.ssl_states(6, 1, K=4, n_opp=0)
    w = dict(PARAMS, w_angle=0.0, w_dist=0.0)
    grid = _grid(12.0, 9.0, 1.0, o)
    out = orc.search(b, grid, [3.0, 6.5], w, dense=True)
    feas = out["feasible"][0].reshape(-1).astype(bool)
    assert feas.any()
    assert out["best_idx"][0] == int(np.flatnonzero(feas)[0])
    assert out["best_score"][0] == w["w_margin"] * w["margin_cap"]


def check_search_reachability(o=None):
    """Without opponents every pass the ball can reach is feasible, and the
    reachable set is the disc of radius v^2 / (2 a) around the ball."""
    orc = _orc(o)
    b = synth.ssl_states(7, 1, K=4, n_opp=0)
    grid = _grid(12.0, 9.0, 0.25, o)
    out = orc.search(b, grid, [2.0], PARAMS, dense=True)
    g, nx, ny, x0, y0 = grid
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    cx, cy = x0 + ix * g, y0 + iy * g
    D = np.hypot(cx - float(b["ball"][0, 0]), cy - float(b["ball"][0, 1]))
    inside = (D <= 4.0 - 1e-9).reshape(-1)
    outside = (D >= 4.0 + 1e-9).reshape(-1)
    feas = out["feasible"][0, 0].astype(bool)
    assert np.all(feas[inside]) and not np.any(feas[outside])
    assert np.all(np.isneginf(out["margin"][0, 0][outside]))


def test_search_consistency():
    check_search_consistency()


def test_search_tie_rule():
    check_search_tie_rule()


def test_search_reachability():
    check_search_reachability()


def test_marked_layout_has_fewer_feasible_passes():
    """Sec. 4.3 observes few feasible points when receivers are marked and
    many when nobody is marked; the marked layout shows the same trend."""
    grid = _grid(12.0, 9.0, 0.5)
    free = synth.ssl_states(21, 6, K=16)
    marked = synth.ssl_states(21, 6, K=16, marked=True)
    none = synth.ssl_states(21, 6, K=16, n_opp=0)
    sp = [3.5, 5.0]
    nf = [oracle.search(b, grid, sp, PARAMS)["n_feasible"].sum()
          for b in (none, free, marked)]
    assert nf[0] > nf[1] > 0 and nf[0] > nf[2]
