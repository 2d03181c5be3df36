"""Seeded synthetic game states shaped like RoboCup SSL play.

This module only draws inputs; it holds none of the search's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  All arrays are
float32 (int32 for counts), the precision the search takes its inputs in.

Recipe (the paper's match logs are not available; uniform states stand in):
  * ball and every robot: position uniform over the field rectangle
    [-L/2, L/2] x [-W/2, W/2];
  * robot velocity: speed uniform in [0, vmax], heading uniform in [0, 2 pi);
  * optional "marked" layout: each opponent placed U[0.3, 1.0] m from a
    random teammate in a uniform direction (clipped to the field), the
    crowded regime the paper describes for surrounded receivers;
  * generator: numpy PCG64 with a fixed seed per workload, draws in a fixed
    order, so a (seed, sizes) pair always gives the same batch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np

# Value-function and feasibility parameters.  The paper states that the
# weights are tuned by hand and gives no values; these are the defaults of
# the build (weights 1, margin capped at 1 s, no safety threshold).  Robot
# radius 0.09 m and goal widths are SSL rule values.
DEFAULT_PARAMS = {
    "w_angle": 1.0,
    "w_dist": 1.0,
    "w_margin": 1.0,
    "margin_cap": 1.0,
    "tau_safe": 0.0,
    "robot_radius": 0.09,
    "reach_radius": 0.0,
    "min_pass_dist": 0.0,
}

GOAL_WIDTH = {(12.0, 9.0): 1.8, (9.0, 6.0): 1.0}


def ssl_states(seed: int, n_states: int, *, field_len: float = 12.0,
               field_wid: float = 9.0, goal_width: float | None = None,
               n_opp: int = 8, j_stride: int | None = None, n_team: int = 8,
               K: int = 64, ball_decel: float = 0.5, vmax: float = 3.25,
               amax: float = 3.0, marked: bool = False) -> dict:
    """A batch of ``n_states`` states with identical shape parameters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _draw(rng, n_states, field_len, field_wid, goal_width, n_opp,
                 j_stride or n_opp, n_team, K, ball_decel, vmax, amax, marked)


def _draw(rng, S, L, W, gw, J, jstride, nteam, K, decel, vmax, amax, marked):
    if gw is None:
        gw = GOAL_WIDTH.get((float(L), float(W)), 1.8)
    lo = np.array([-L / 2, -W / 2])
    hi = np.array([L / 2, W / 2])
    ball = rng.uniform(lo, hi, size=(S, 2))
    team = rng.uniform(lo, hi, size=(S, nteam, 2))
    tspeed = rng.uniform(0.0, vmax, size=(S, nteam))
    thead = rng.uniform(0.0, 2 * math.pi, size=(S, nteam))
    opp = rng.uniform(lo, hi, size=(S, J, 2))
    ospeed = rng.uniform(0.0, vmax, size=(S, J))
    ohead = rng.uniform(0.0, 2 * math.pi, size=(S, J))
    if marked and nteam > 0:
        mate = rng.integers(0, nteam, size=(S, J))
        dist = rng.uniform(0.3, 1.0, size=(S, J))
        ang = rng.uniform(0.0, 2 * math.pi, size=(S, J))
        base = np.take_along_axis(team, mate[..., None], axis=1)
        off = np.stack([dist * np.cos(ang), dist * np.sin(ang)], axis=-1)
        opp = np.clip(base + off, lo, hi)
    opp_pos = np.zeros((S, jstride, 2), np.float32)
    opp_vel = np.zeros((S, jstride, 2), np.float32)
    opp_pos[:, :J] = opp
    opp_vel[:, :J, 0] = ospeed * np.cos(ohead)
    opp_vel[:, :J, 1] = ospeed * np.sin(ohead)
    team_vel = np.stack([tspeed * np.cos(thead), tspeed * np.sin(thead)], -1)
    full = lambda x, dt=np.float32: np.full(S, x, dt)  # noqa: E731
    return {
        "ball": ball.astype(np.float32),
        "n_opp": full(J, np.int32),
        "opp_pos": opp_pos,
        "opp_vel": opp_vel,
        "team_pos": team.astype(np.float32),
        "team_vel": team_vel.astype(np.float32),
        "ball_decel": full(decel),
        "vmax": full(vmax),
        "amax": full(amax),
        "field_len": full(L),
        "field_wid": full(W),
        "goal_width": full(gw),
        "K": full(K, np.int32),
    }


def concat(batches: list[dict]) -> dict:
    """Concatenate batches along the state axis (padding opponent slots)."""
    J = max(b["opp_pos"].shape[1] for b in batches)
    out = {}
    for k in batches[0]:
        parts = []
        for b in batches:
            x = b[k]
            if k in ("opp_pos", "opp_vel") and x.shape[1] < J:
                pad = np.zeros((x.shape[0], J - x.shape[1], 2), x.dtype)
                x = np.concatenate([x, pad], axis=1)
            parts.append(x)
        if k in ("team_pos", "team_vel"):
            T = max(p.shape[1] for p in parts)
            parts = [np.concatenate([p, np.zeros((p.shape[0], T - p.shape[1], 2),
                                                 p.dtype)], axis=1)
                     if p.shape[1] < T else p for p in parts]
        out[k] = np.concatenate(parts, axis=0)
    return out


def take(batch: dict, idx) -> dict:
    """Sub-batch of the states ``idx``."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in batch.items()}


@dataclass
class Workload:
    """A named workload: states plus the shared grid spacing and speeds."""
    name: str
    seed: int
    n_states: int
    spacing: float
    speeds: list
    K: int
    field: tuple = (12.0, 9.0)
    n_opp: int = 8
    ball_decel: float = 0.5
    vmax: float = 3.25
    amax: float = 3.0
    params: dict = dc_field(default_factory=lambda: dict(DEFAULT_PARAMS))

    def states(self, n_states: int | None = None, marked=False) -> dict:
        return ssl_states(self.seed, self.n_states if n_states is None
                          else n_states, field_len=self.field[0],
                          field_wid=self.field[1], n_opp=self.n_opp, K=self.K,
                          ball_decel=self.ball_decel, vmax=self.vmax,
                          amax=self.amax, marked=marked)

    def speeds_f32(self):
        return np.asarray(self.speeds, np.float32)


# Plain exact search of one state: 12x9 m, 0.1 m grid (121x91), one kick
# speed 4 m/s, K = 32, decel 0.5, 8 v 8, vmax 3.25, amax 3.
SINGLE = Workload("single_12x9_g0.1_v1_K32_J8", seed=0, n_states=1,
                  spacing=0.1, speeds=[4.0], K=32)

# Batched exact search: 4096 states, 12x9 m, 0.05 m grid (241x181), speeds
# {2, 3.5, 5, 6.5} m/s, K = 64, 8 v 8.
BATCHED = Workload("batched_4096x241x181_v4_K64_J8", seed=1, n_states=4096,
                   spacing=0.05, speeds=[2.0, 3.5, 5.0, 6.5], K=64)


# Learned-proposal workload: 4096 states of the batched kind (12x9 m, 8 v 8,
# K = 64, speeds {2, 3.5, 5, 6.5}) searched on the 0.025 m grid (481x361),
# plain and through the proposal.  Seed 7 is held out of the network's
# training set (seeds 100000 and up).
PROPOSAL = Workload("proposal_4096x481x361_v4_K64_J8", seed=7, n_states=4096,
                    spacing=0.025, speeds=[2.0, 3.5, 5.0, 6.5], K=64)


# The paper's own search parameterisation (directions x kick powers,
# Sec. 4.2): 12x9 m, 16 receivers and 16 opponents (the paper's 32 robots on
# the field), K = 64 samples per ball path, 128 directions x 64 kick powers
# in [1, 6.5] m/s; the ball at the passer's feet.
DPPS_SEED = 5
DPPS_STATES = 4096
DPPS_PARAMS = {"n_dir": 128, "n_pow": 64, "v_lo": 1.0, "v_hi": 6.5,
               "slide": 5.0 / 7.0, "tau_delta": 0.0, "delta_cap": 1.0,
               "w_time": 1.0, "w_angle": 1.0, "w_dist": 1.0, "w_refr": 1.0,
               "w_delta": 1.0, "robot_radius": 0.09, "reach_radius": 0.0}


def dpps_states(seed: int, n_states: int, *, n_team: int = 16,
                n_opp: int = 16, K: int = 64) -> dict:
    """States with receivers (team_pos, team_vel) for the direction x power
    search: uniform positions, speeds U[0, vmax], uniform headings."""
    b = ssl_states(seed, n_states, n_opp=n_opp, n_team=n_team, K=K)
    b["n_team"] = np.full(n_states, n_team, np.int32)
    return b


def dpps_oracle_params(p: dict = DPPS_PARAMS) -> dict:
    """The same parameters under the oracle's names."""
    return {"vlo": p["v_lo"], "vhi": p["v_hi"], "slide": p["slide"],
            "tau_delta": p["tau_delta"], "delta_cap": p["delta_cap"],
            "w_time": p["w_time"], "w_angle": p["w_angle"],
            "w_dist": p["w_dist"], "w_refr": p["w_refr"],
            "w_delta": p["w_delta"], "robot_radius": p["robot_radius"],
            "reach_radius": p["reach_radius"], "min_time": 0.0}


# Running points (Sec. 5.1-5.2).  The paper gives no weights and no
# criterion constants; these defaults are the build's: the 0.1 m raster the
# paper names, weights 1, full distance credit from 2 m off the ball, full
# angle credit 0.25-0.75 rad off the goal axis (falling to 0 over 0.5 rad),
# the 2019 SSL division-A defence area (1.2 m deep, 2.4 m wide), guard times
# capped at 2 s, four supporters.
RUN_SEED = 6
RUN_STATES = 4096
RUN_PARAMS = {"spacing": 0.1, "w_goal": 1.0, "w_ball": 1.0, "w_angle": 1.0,
              "w_guard": 1.0, "w_avoid": 1.0, "ball_ref": 2.0,
              "angle_lo": 0.25, "angle_hi": 0.75, "angle_span": 0.5,
              "def_depth": 1.2, "def_width": 2.4, "guard_cap": 2.0,
              "n_run": 4}


def run_states(seed: int, n_states: int, *, n_opp: int = 16,
               def_depth: float = 1.2, def_width: float = 2.4) -> dict:
    """States for the running-point search: as ``dpps_states``, but the
    first opponent is a goalkeeper, placed uniformly inside the defence area
    of the goal at +L/2, and in half the states (drawn) the second opponent
    is a second guard placed the same way."""
    b = dpps_states(seed, n_states, n_team=0, n_opp=n_opp, K=1)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    L = b["field_len"].astype(np.float64)
    for j in range(min(2, n_opp)):
        x = 0.5 * L - rng.uniform(0.0, def_depth, n_states)
        y = rng.uniform(-0.5 * def_width, 0.5 * def_width, n_states)
        take = np.ones(n_states, bool) if j == 0 else \
            rng.uniform(size=n_states) < 0.5
        b["opp_pos"][take, j, 0] = x[take]
        b["opp_pos"][take, j, 1] = y[take]
    return b


def run_oracle_params(p: dict = RUN_PARAMS) -> dict:
    """The running-point parameters as the CUDA path holds them (float32),
    promoted for the oracle."""
    return {k: (float(np.float32(v)) if k != "n_run" else int(v))
            for k, v in p.items()}


def uneven_batch(seed: int, n_states: int, *,
                 spacings=(0.025, 0.05, 0.1), k_range=(32, 128),
                 speed_range=(2.0, 6.5), decel_range=(0.3, 0.7),
                 vmax: float = 3.25, amax: float = 3.0) -> dict:
    """An uneven batch: half the states on a 12 x 9 m field with 11
    opponents, half on 9 x 6 m with 6; per state a grid spacing drawn from
    ``spacings``, 1-8 kick speeds uniform in ``speed_range`` (sorted), K
    uniform in ``k_range`` and a ball deceleration uniform in
    ``decel_range``.  Opponent slots are padded to 16.  Besides the state
    arrays of ``ssl_states`` it holds ``spacing`` (S,), ``n_speeds`` (S,) and
    ``speeds`` (S, 8; unused slots 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = n_states
    big = rng.integers(0, 2, S) == 0
    L = np.where(big, 12.0, 9.0)
    W = np.where(big, 9.0, 6.0)
    gw = np.where(big, 1.8, 1.0)
    J = np.where(big, 11, 6).astype(np.int32)
    spacing = rng.choice(np.asarray(spacings, np.float64), S)
    n_speeds = rng.integers(1, 9, S).astype(np.int32)
    sp = np.sort(rng.uniform(speed_range[0], speed_range[1], (S, 8)), axis=1)
    speeds = np.where(np.arange(8)[None, :] < n_speeds[:, None], sp, 0.0)
    K = rng.integers(k_range[0], k_range[1] + 1, S).astype(np.int32)
    decel = rng.uniform(decel_range[0], decel_range[1], S)
    half = np.stack([L / 2, W / 2], axis=1)
    ball = rng.uniform(-1.0, 1.0, (S, 2)) * half
    opp = rng.uniform(-1.0, 1.0, (S, 16, 2)) * half[:, None, :]
    ospeed = rng.uniform(0.0, vmax, (S, 16))
    ohead = rng.uniform(0.0, 2 * math.pi, (S, 16))
    used = np.arange(16)[None, :] < J[:, None]
    opp_pos = np.where(used[..., None], opp, 0.0)
    opp_vel = np.where(used[..., None],
                       np.stack([ospeed * np.cos(ohead),
                                 ospeed * np.sin(ohead)], -1), 0.0)
    f32 = np.float32
    return {
        "ball": ball.astype(f32),
        "n_opp": J,
        "opp_pos": opp_pos.astype(f32),
        "opp_vel": opp_vel.astype(f32),
        "ball_decel": decel.astype(f32),
        "vmax": np.full(S, vmax, f32),
        "amax": np.full(S, amax, f32),
        "field_len": L.astype(f32),
        "field_wid": W.astype(f32),
        "goal_width": gw.astype(f32),
        "K": K,
        "spacing": spacing.astype(f32),
        "n_speeds": n_speeds,
        "speeds": speeds.astype(f32),
    }


# Uneven batch + autotuner: 8192 states mixing 12x9 m / 11 v 11 and
# 9x6 m / 6 v 6, grids 0.025-0.1 m, 1-8 kick speeds in [2, 6.5] m/s,
# K 32-128, ball deceleration U[0.3, 0.7] m/s^2.
UNEVEN_SEED = 2
UNEVEN_STATES = 8192


def serving_matches(seed: int, n_matches: int, n_frames: int, *,
                    hz: float = 60.0, spacing: float = 0.05,
                    speeds=(2.0, 3.5, 5.0, 6.5), K: int = 32,
                    vmax: float = 3.25, amax: float = 3.0,
                    ball_decel: float = 0.5) -> dict:
    """Simulated matches for the serving loop.  Each match plays on a 12 x 9
    or 9 x 6 m field with 6-11 opponents; its frames are 1/hz apart, robots
    moving with a random acceleration of at most amax per axis, speed capped
    at vmax, reflected at the field edges; the ball drifts the same way at
    half the speed.  Returns state arrays of shape (n_matches * n_frames,
    ...) in match-major order plus per-match ``field_len``, ``field_wid``,
    ``n_opp_match`` and the shared ``spacing`` and ``speeds``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M, F = n_matches, n_frames
    big = rng.integers(0, 2, M) == 0
    L = np.where(big, 12.0, 9.0)
    W = np.where(big, 9.0, 6.0)
    J = rng.integers(6, 12, M).astype(np.int32)
    half = np.stack([L / 2, W / 2], axis=1)            # (M, 2)
    dt = 1.0 / hz
    pos = rng.uniform(-1, 1, (M, 16, 2)) * half[:, None, :]
    vel = rng.uniform(-1, 1, (M, 16, 2)) * vmax / math.sqrt(2)
    ball = rng.uniform(-1, 1, (M, 2)) * half
    bvel = rng.uniform(-1, 1, (M, 2)) * vmax / 2
    out_pos = np.zeros((M, F, 16, 2))
    out_vel = np.zeros((M, F, 16, 2))
    out_ball = np.zeros((M, F, 2))
    for f in range(F):
        out_pos[:, f], out_vel[:, f], out_ball[:, f] = pos, vel, ball
        vel = vel + rng.uniform(-amax, amax, vel.shape) * dt
        sp = np.linalg.norm(vel, axis=-1, keepdims=True)
        vel = np.where(sp > vmax, vel * (vmax / np.maximum(sp, 1e-9)), vel)
        pos = pos + vel * dt
        over = np.abs(pos) > half[:, None, :]
        vel = np.where(over, -vel, vel)
        pos = np.clip(pos, -half[:, None, :], half[:, None, :])
        bvel = bvel + rng.uniform(-amax, amax, bvel.shape) * dt / 2
        ball = np.clip(ball + bvel * dt, -half, half)
    used = np.arange(16)[None, None, :] < J[:, None, None]
    S = M * F
    f32 = np.float32
    rep = lambda a: np.repeat(a, F)  # noqa: E731  per-match -> per-frame
    return {
        "ball": out_ball.reshape(S, 2).astype(f32),
        "n_opp": rep(J).astype(np.int32),
        "opp_pos": np.where(used[..., None], out_pos, 0).reshape(S, 16, 2)
        .astype(f32),
        "opp_vel": np.where(used[..., None], out_vel, 0).reshape(S, 16, 2)
        .astype(f32),
        "ball_decel": np.full(S, ball_decel, f32),
        "vmax": np.full(S, vmax, f32),
        "amax": np.full(S, amax, f32),
        "field_len": rep(L).astype(f32),
        "field_wid": rep(W).astype(f32),
        "goal_width": rep(np.where(big, 1.8, 1.0)).astype(f32),
        "K": np.full(S, K, np.int32),
        "spacing": np.full(S, spacing, f32),
        "n_speeds": np.full(S, len(speeds), np.int32),
        "speeds": np.tile(np.pad(np.asarray(speeds, f32),
                                 (0, 8 - len(speeds))), (S, 1)),
        "n_matches": M,
        "n_frames": F,
    }


# Serving: 512 concurrent simulated matches at 60 Hz, 9x6 or 12x9 fields,
# 6-11 opponents, grid 0.05 m, 4 kick speeds (K = 32 samples per pass).
SERVING_SEED = 4
SERVING_MATCHES = 512


# Input maps of the proposal network (46 x 61 pixels x 8 channels), drawn
# directly instead of rasterised from states, for checking the network's
# kernels on the same input on both sides.  Each channel is uniform over
# the range the rasteriser's channel takes on a 12 x 9 m field (opponent
# density, coarse score with a share of cells at the floor, ball distance,
# margin, shot angle / pi, goal distance, x and y); the low 16 bits of every
# float32 are cleared, so each value is exactly a bfloat16 (returned as its
# 16-bit pattern).
NET_MAP_RANGES = ((0.0, 2.0), (-1.1, 1.5), (0.0, 1.0), (-2.0, 1.0),
                  (0.0, 0.35), (0.0, 1.0), (-1.0, 1.0), (-1.0, 1.0))
NET_MAP_FLOOR = -1.2      # the coarse score where no pass is feasible
NET_MAP_FLOOR_SHARE = 0.3


def net_maps(seed: int, n: int, h: int = 46, w: int = 61,
             integer: bool = False) -> np.ndarray:
    """n seeded input maps, uint16 bfloat16 patterns of shape (n, h, w, 8).
    integer: every value an integer in 0..3 instead (with integer weights
    the network's sums are then exact in float32 and bfloat16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if integer:
        x = rng.integers(0, 4, size=(n, h, w, 8)).astype(np.float32)
        return (x.view(np.uint32) >> 16).astype(np.uint16)
    lo = np.array([r[0] for r in NET_MAP_RANGES])
    hi = np.array([r[1] for r in NET_MAP_RANGES])
    x = rng.uniform(lo, hi, size=(n, h, w, 8)).astype(np.float32)
    floor = rng.uniform(size=(n, h, w)) < NET_MAP_FLOOR_SHARE
    x[..., 1] = np.where(floor, np.float32(NET_MAP_FLOOR), x[..., 1])
    return (x.view(np.uint32) >> 16).astype(np.uint16)


NET_LAYERS = ((8, 32), (32, 32), (32, 32), (32, 1))   # (inputs, outputs)


def net_int_weights(seed: int, nonzero: int = 3) -> np.ndarray:
    """Integer weights for the proposal network, flat in the library's
    layout (per layer W[3][3][cout][cin], then bias[cout]): each output
    channel of a hidden layer takes `nonzero` taps of weight +-1 -- the
    first on input channel (c mod cin) through a permutation, so that every
    input channel feeds some output, the others at random -- the rest 0;
    the output channel takes one +-1 tap on every input channel; biases are
    integers in -1..1.  On integer input maps every sum stays a small
    integer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for ci, co in NET_LAYERS:
        W = np.zeros((9, co, ci), np.float32)
        perm = rng.permutation(max(ci, co))
        for c in range(co):
            if co == 1:
                taps = rng.integers(0, 9, size=ci)
                W[taps, c, np.arange(ci)] = rng.choice([-1.0, 1.0], size=ci)
                continue
            first = perm[c] % ci
            rest = rng.choice(9 * ci, size=nonzero - 1, replace=False)
            W[rng.integers(0, 9), c, first] = rng.choice([-1.0, 1.0])
            W[rest // ci, c, rest % ci] = rng.choice([-1.0, 1.0],
                                                     size=nonzero - 1)
        out += [W.reshape(-1), rng.integers(-1, 2, size=co).astype(np.float32)]
    return np.concatenate(out)


def serving_states(seed: int, n_states: int, *, K: int = 32,
                   vmax: float = 3.25, amax: float = 3.0,
                   ball_decel: float = 0.5) -> dict:
    """Independent states shaped like the serving frames: half on a 12 x 9 m
    field and half on a 9 x 6 m one (interleaved), 6-11 opponents each
    (uniform), positions uniform over the field, speeds uniform in
    [0, vmax], K samples.  Opponent slots past n_opp hold drawn values the
    search ignores."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for L, W in ((12.0, 9.0), (9.0, 6.0)):
        n = (n_states + (L == 12.0)) // 2
        b = _draw(rng, n, L, W, None, 11, 16, 8, K, ball_decel, vmax, amax,
                  False)
        b["n_opp"] = rng.integers(6, 12, n).astype(np.int32)
        parts.append(b)
    big, small = parts
    order = np.empty(n_states, np.int64)
    order[0::2] = np.arange(big["ball"].shape[0])
    order[1::2] = big["ball"].shape[0] + np.arange(small["ball"].shape[0])
    return take(concat([big, small]), order)
