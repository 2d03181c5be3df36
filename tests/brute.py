"""Brute-force references used to pin the oracle (tests only).

These do not solve any closed form: the ball and the robots are stepped
forward in time at a fixed step (1 ms by default) and the first step at
which the target is reached is reported, so each result is within one step
of the exact time.  Geometry for the shot angle is checked by casting rays.
They share no code with ``oracle/`` or with the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np


def ball_arrival_sim(s, v, a, dt=1e-3, t_max=60.0):
    """Time-step a ball rolling from speed v with deceleration a; return the
    first step time at which it has covered s (inf if it stops first).
    Vectorised over numpy arrays of equal shape."""
    s, v, a = np.broadcast_arrays(np.asarray(s, float), np.asarray(v, float),
                                  np.asarray(a, float))
    x = np.zeros(s.shape)
    vel = v.copy()
    t_hit = np.full(s.shape, np.inf)
    t_hit[s <= 0] = 0.0
    t = 0.0
    n = int(t_max / dt)
    for i in range(1, n + 1):
        live = ~np.isfinite(t_hit) & (vel > 0)
        if not live.any():
            break
        # Within one step the speed drops linearly (rolling friction), so the
        # distance covered is the step's mean speed times dt.
        vnew = np.maximum(vel - a * dt, 0.0)
        x = x + 0.5 * (vel + vnew) * dt
        vel = vnew
        t = i * dt
        hit = live & (x >= s)
        t_hit[hit] = t
    return t_hit


def robot_arrival_sim_1d(d, w, vmax, amax, dt=1e-3, t_max=60.0):
    """1-D robot starting at 0 with velocity w (toward +), accelerating at
    amax toward +d, speed capped at vmax; first step time with x >= d."""
    d, w = np.broadcast_arrays(np.asarray(d, float), np.asarray(w, float))
    x = np.zeros(d.shape)
    vel = np.clip(w, -vmax, vmax).astype(float)
    t_hit = np.where(d <= 0, 0.0, np.inf)
    n = int(t_max / dt)
    for i in range(1, n + 1):
        live = ~np.isfinite(t_hit)
        if not live.any():
            break
        vnew = np.minimum(vel + amax * dt, vmax)
        # Speed is piecewise linear inside the step (ramp, then flat).
        x = x + 0.5 * (vel + vnew) * dt
        vel = vnew
        hit = live & (x >= d)
        t_hit[hit] = i * dt
    return t_hit


def robot_arrival_sim(o, u, p, vmax, amax, reach=0.0, dt=1e-3):
    """2-D robot at o with velocity u heading for p.  The robot moves along
    the line o->p with the velocity component toward p as its initial speed
    (the perpendicular part is dropped) and stops as soon as its centre is
    within ``reach`` of p."""
    o, u, p = (np.asarray(x, float) for x in (o, u, p))
    diff = p - o
    d = math.hypot(diff[0], diff[1])
    if d <= reach:
        return 0.0
    e = diff / d
    w = float(u[0] * e[0] + u[1] * e[1])
    return float(robot_arrival_sim_1d(d - reach, w, vmax, amax, dt))


def candidate_margin_sim(ball, opps, c, v, decel, vmax, amax, K, reach=0.0,
                         dt=1e-3):
    """Margin of the pass from ``ball`` to ``c`` by stepping every robot and
    the ball to each of the K sample points: min_k (T_k - t_ball_k).
    ``opps``: list of (pos, vel).  Returns (margin, [T_k], [t_ball_k])."""
    b = np.asarray(ball, float)
    c = np.asarray(c, float)
    D = math.hypot(*(c - b))
    Ts, tbs = [], []
    m = math.inf
    for k in range(1, K + 1):
        frac = k / K
        pk = b + frac * (c - b)
        T = math.inf
        for (op, ov) in opps:
            T = min(T, robot_arrival_sim(op, ov, pk, vmax, amax, reach, dt))
        tb = float(ball_arrival_sim(frac * D, v, decel, dt))
        Ts.append(T)
        tbs.append(tb)
        m = min(m, T - tb)
    return m, Ts, tbs


def shot_angle_rays(c, opps_xy, L, gw, r, n_rays=100_000):
    """Largest run of unobstructed rays from c into the goal mouth, times the
    angular step.  A ray is obstructed when an opponent disc of radius r
    intersects it (closest approach of the disc centre to the ray <= r)."""
    c = np.asarray(c, float)
    gx = L / 2
    lo = math.atan2(-gw / 2 - c[1], gx - c[0])
    hi = math.atan2(gw / 2 - c[1], gx - c[0])
    step = (hi - lo) / n_rays
    ang = lo + (np.arange(n_rays) + 0.5) * step
    e = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    blocked = np.zeros(n_rays, bool)
    for (ox, oy) in opps_xy:
        rel = np.array([ox, oy]) - c
        along = e @ rel
        perp = np.abs(e[:, 0] * rel[1] - e[:, 1] * rel[0])
        dist = np.where(along >= 0, perp, math.hypot(*rel))
        blocked |= dist <= r
    best = run = 0
    for b in blocked:
        run = 0 if b else run + 1
        best = max(best, run)
    return best * step, step
