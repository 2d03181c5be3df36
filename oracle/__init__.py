"""FP64 CPU oracle for the passing-point search (ZJUNlict 2019, Sec. 4.1-4.4)
and the running points (Sec. 5.1-5.2).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  It shares no code with the CUDA path: it takes plain float64
arrays, defines its own grid rule and loads its own C library
(``pps_oracle.c``, compiled with gcc, no fast-math).

Every function here is a thin ctypes marshaller; the arithmetic is in
``pps_oracle.c``, whose header comment lists the readings of the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pps_oracle.c")
_HDR = os.path.join(_HERE, "pps_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()

# Scalar record and parameter layouts (pps_oracle.h).
SCALARS = ("ball_x", "ball_y", "ball_decel", "vmax", "amax",
           "field_len", "field_wid", "goal_width")
PARAMS = ("w_angle", "w_dist", "w_margin", "margin_cap", "tau_safe",
          "robot_radius", "reach_radius", "min_pass_dist")
# Parameters of the direction x power search (pps_oracle.h, PPS_ORACLE_D_*).
DPPS_PARAMS = ("vlo", "vhi", "slide", "tau_delta", "delta_cap", "w_time",
               "w_angle", "w_dist", "w_refr", "w_delta", "robot_radius",
               "reach_radius", "min_time")
# Running-point parameters, in the order of PPS_ORACLE_R_* (pps_oracle.h).
RUN_PARAMS = ("spacing", "w_goal", "w_ball", "w_angle", "w_guard", "w_avoid",
              "ball_ref", "angle_lo", "angle_hi", "angle_span", "def_depth",
              "def_width", "guard_cap", "n_run")
RUN_CRITERIA = ("goal", "ball", "angle", "guard", "avoid")


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle library (gcc -O2 -fopenmp, no fast-math)."""
    hdr_dir = os.path.dirname(os.path.abspath(src))
    stale = (not os.path.exists(out)
             or os.path.getmtime(out) < max(os.path.getmtime(src),
                                            os.path.getmtime(_HDR)))
    if force or stale:
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-Wall", "-Wextra", "-I", _HERE, "-I", hdr_dir, "-o", tmp, src,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _bind(lib):
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    lib.pps_oracle_ball_time.restype = d
    lib.pps_oracle_ball_time.argtypes = [d, d, d]
    lib.pps_oracle_intercept_time.restype = d
    lib.pps_oracle_intercept_time.argtypes = [d] * 9
    lib.pps_oracle_min_intercept.restype = d
    lib.pps_oracle_min_intercept.argtypes = [p, d, d, d]
    lib.pps_oracle_min_intercept_many.restype = None
    lib.pps_oracle_min_intercept_many.argtypes = [p, i, p, d, p]
    lib.pps_oracle_margin.restype = d
    lib.pps_oracle_margin.argtypes = [p, d, d, d, d, p, p]
    lib.pps_oracle_shot_angle.restype = d
    lib.pps_oracle_shot_angle.argtypes = [p, d, d, d]
    lib.pps_oracle_score.restype = d
    lib.pps_oracle_score.argtypes = [p, p, d, d, d]
    lib.pps_oracle_grid.restype = None
    lib.pps_oracle_grid.argtypes = [d, d, d, p, p, p, p]
    lib.pps_oracle_search.restype = i
    lib.pps_oracle_search.argtypes = (
        [i, p, p, p, i, p, d, i, i, d, d, p, i, p] + [p] * 8 + [i, i])
    lib.pps_oracle_max_threads.restype = i
    lib.pps_oracle_max_threads.argtypes = []
    lib.pps_oracle_dpps_path.restype = d
    lib.pps_oracle_dpps_path.argtypes = [p, d, d, d, p]
    lib.pps_oracle_dpps_group.restype = d
    lib.pps_oracle_dpps_group.argtypes = [p, i, p, d, d, d, d, p, p]
    lib.pps_oracle_dpps_candidate.restype = None
    lib.pps_oracle_dpps_candidate.argtypes = [p, p, i, i, i, i, p]
    lib.pps_oracle_pass_power.restype = None
    lib.pps_oracle_pass_power.argtypes = [p, i, d, d, d, d, d, d, d, p]
    lib.pps_oracle_shoot.restype = None
    lib.pps_oracle_shoot.argtypes = [p, d, d, d, d, d, d, d, d, p]
    lib.pps_oracle_shot_gap.restype = d
    lib.pps_oracle_shot_gap.argtypes = [p, d, d, d, p]
    lib.pps_oracle_dpps_search.restype = i
    lib.pps_oracle_dpps_search.argtypes = [i, p, p, p, p, p, p, i, i, i, p,
                                           p, p, p, p, p, p, p, i]
    lib.pps_oracle_run_point.restype = None
    lib.pps_oracle_run_point.argtypes = [p, p, d, d, p]
    lib.pps_oracle_run_zone.restype = i
    lib.pps_oracle_run_zone.argtypes = [p, p, d, d]
    lib.pps_oracle_run_choose.restype = None
    lib.pps_oracle_run_choose.argtypes = [p, p, i, i, p]
    lib.pps_oracle_run_search.restype = i
    lib.pps_oracle_run_search.argtypes = [i, p, p, p, i, p, p, p, p, p, p, p,
                                          i]
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _State(ctypes.Structure):
    _fields_ = [("sc", ctypes.c_void_p), ("n_opp", ctypes.c_int),
                ("opp", ctypes.c_void_p), ("K", ctypes.c_int)]


class State:
    """One state in the oracle's own layout (all float64).

    ``scalars``: dict with the keys of ``SCALARS``; ``opp``: (n, 4) array of
    x, y, vx, vy; ``K``: samples per pass line.
    """

    def __init__(self, scalars: dict, opp, K: int):
        self.sc = np.array([float(scalars[k]) for k in SCALARS], np.float64)
        self.opp = np.ascontiguousarray(
            np.asarray(opp, np.float64).reshape(-1, 4))
        self.K = int(K)
        self._c = _State(_ptr(self.sc), self.opp.shape[0], _ptr(self.opp),
                         self.K)

    @property
    def ref(self):
        return ctypes.byref(self._c)


class Oracle:
    """The oracle's entry points over one loaded copy of the C library.

    ``Oracle()`` uses ``pps_oracle.c``; ``Oracle(path)`` loads another build
    of it (the tests load deliberately broken copies to show that the pins
    catch them)."""

    def __init__(self, lib_path: str | None = None):
        self.lib = _bind(ctypes.CDLL(lib_path or build()))

    def grid(self, L, W, g):
        """Grid rule of the oracle: (nx, ny, x0, y0)."""
        nx, ny = ctypes.c_int(), ctypes.c_int()
        x0, y0 = ctypes.c_double(), ctypes.c_double()
        self.lib.pps_oracle_grid(float(L), float(W), float(g),
                                 ctypes.byref(nx), ctypes.byref(ny),
                                 ctypes.byref(x0), ctypes.byref(y0))
        return nx.value, ny.value, x0.value, y0.value

    def ball_time(self, s, v, a):
        return self.lib.pps_oracle_ball_time(float(s), float(v), float(a))

    def intercept_time(self, o, u, p, vmax, amax, reach=0.0):
        return self.lib.pps_oracle_intercept_time(
            float(o[0]), float(o[1]), float(u[0]), float(u[1]), float(p[0]),
            float(p[1]), float(vmax), float(amax), float(reach))

    def min_intercept(self, state: State, p, reach=0.0):
        return self.lib.pps_oracle_min_intercept(state.ref, float(p[0]),
                                                 float(p[1]), float(reach))

    def min_intercept_many(self, state: State, pts, reach=0.0):
        """min_intercept at each row of the (n, 2) array ``pts``."""
        pts = np.ascontiguousarray(np.asarray(pts, np.float64).reshape(-1, 2))
        out = np.empty(pts.shape[0], np.float64)
        self.lib.pps_oracle_min_intercept_many(state.ref, pts.shape[0],
                                               _ptr(pts), float(reach),
                                               _ptr(out))
        return out

    def margin(self, state: State, c, v, reach=0.0):
        """(margin, reachable, T[K]) of the pass to point c at speed v."""
        T = np.empty(state.K, np.float64)
        r = ctypes.c_int()
        m = self.lib.pps_oracle_margin(state.ref, float(c[0]), float(c[1]),
                                       float(v), float(reach), _ptr(T),
                                       ctypes.byref(r))
        return m, bool(r.value), T

    def shot_angle(self, state: State, c, r):
        return self.lib.pps_oracle_shot_angle(state.ref, float(c[0]),
                                              float(c[1]), float(r))

    def score(self, state: State, params: dict, c, m):
        prm = np.array([float(params[k]) for k in PARAMS], np.float64)
        return self.lib.pps_oracle_score(state.ref, _ptr(prm), float(c[0]),
                                         float(c[1]), float(m))

    def search(self, batch: dict, grid_spec, speeds, params: dict, *,
               dense=False, want_T=False, n_threads=0):
        """Run the oracle over a batch.

        ``batch``: arrays of a seeded input batch (promoted to float64):
        ball (S,2), n_opp (S,), opp_pos (S,J,2), opp_vel (S,J,2), ball_decel,
        vmax, amax, field_len, field_wid, goal_width (S,), K (S,).
        ``grid_spec``: (g, nx, ny, x0, y0).  Returns a dict of numpy arrays.
        """
        ball = np.asarray(batch["ball"], np.float64)
        S = ball.shape[0]
        sc = np.stack([ball[:, 0], ball[:, 1]]
                      + [np.asarray(batch[k], np.float64)
                         for k in SCALARS[2:]], axis=1)
        sc = np.ascontiguousarray(sc)
        opp_pos = np.asarray(batch["opp_pos"], np.float64)
        opp_vel = np.asarray(batch["opp_vel"], np.float64)
        J = opp_pos.shape[1]
        opp = np.ascontiguousarray(np.concatenate([opp_pos, opp_vel], axis=2))
        n_opp = np.ascontiguousarray(np.asarray(batch["n_opp"], np.int32))
        K = np.ascontiguousarray(np.asarray(batch["K"], np.int32))
        g, nx, ny, x0, y0 = grid_spec
        P = int(nx) * int(ny)
        sp = np.ascontiguousarray(np.asarray(speeds, np.float64))
        V = sp.shape[0]
        prm = np.array([float(params[k]) for k in PARAMS], np.float64)
        out = {
            "best_idx": np.empty(S, np.int64),
            "best_score": np.empty(S, np.float64),
            "best_margin": np.empty(S, np.float64),
            "n_feasible": np.empty(S, np.int64),
        }
        kstride = int(K.max()) if S else 1
        if dense:
            out["feasible"] = np.empty((S, V, P), np.uint8)
            out["margin"] = np.empty((S, V, P), np.float64)
            out["score"] = np.empty((S, V, P), np.float64)
        if want_T:
            out["T"] = np.empty((S, P, kstride), np.float64)
        rc = self.lib.pps_oracle_search(
            S, _ptr(sc), _ptr(n_opp), _ptr(K), J, _ptr(opp), float(g),
            int(nx), int(ny), float(x0), float(y0), _ptr(sp), V, _ptr(prm),
            _ptr(out["best_idx"]), _ptr(out["best_score"]),
            _ptr(out["best_margin"]), _ptr(out["n_feasible"]),
            _ptr(out.get("feasible")), _ptr(out.get("margin")),
            _ptr(out.get("score")), _ptr(out.get("T")), kstride,
            int(n_threads))
        if rc != 0:
            raise ValueError("oracle rejected the batch")
        return out

    def max_threads(self) -> int:
        return self.lib.pps_oracle_max_threads()

    # -- direction x power search (pps_oracle.h, D) --
    def dpps_path(self, st: DState, u, v):
        """(path length, stopped) of the ball rolling at v along u."""
        stopped = ctypes.c_int()
        S = self.lib.pps_oracle_dpps_path(st.ref, float(u[0]), float(u[1]),
                                          float(v), ctypes.byref(stopped))
        return S, bool(stopped.value)

    def dpps_group(self, st: DState, robots, u, v, reach=0.0):
        """(time, sample k, robot) of a group's first interception."""
        r = np.ascontiguousarray(np.asarray(robots, np.float64).reshape(-1, 4))
        k, who = ctypes.c_int(), ctypes.c_int()
        t = self.lib.pps_oracle_dpps_group(
            st.ref, r.shape[0], _ptr(r), float(u[0]), float(u[1]), float(v),
            float(reach), ctypes.byref(k), ctypes.byref(who))
        return t, k.value, who.value

    def dpps_candidate(self, st: DState, params: dict, ndir, npow, i, j):
        prm = np.array([float(params[k]) for k in DPPS_PARAMS], np.float64)
        out = np.empty(10, np.float64)
        self.lib.pps_oracle_dpps_candidate(st.ref, _ptr(prm), int(ndir),
                                           int(npow), int(i), int(j),
                                           _ptr(out))
        keys = ("t_team", "t_opp", "k_team", "receiver", "rx", "ry",
                "feasible", "score", "m_team", "m_opp")
        return dict(zip(keys, out.tolist()))

    def pass_power(self, st: DState, receiver, target, buffer=0.3,
                   slide=5 / 7, v_lo=1.0, v_hi=6.5, reach=0.0):
        out = np.empty(5, np.float64)
        self.lib.pps_oracle_pass_power(st.ref, int(receiver), float(target[0]),
                                       float(target[1]), float(buffer),
                                       float(slide), float(v_lo), float(v_hi),
                                       float(reach), _ptr(out))
        return dict(zip(("v0", "v1", "t_pass", "t_recv", "clamped"),
                        out.tolist()))

    def shoot(self, st: DState, c, v_shot=6.5, slide=5 / 7, theta_min=0.1,
              tau=0.0, robot_radius=0.09, reach=0.0):
        out = np.empty(6, np.float64)
        self.lib.pps_oracle_shoot(st.ref, float(c[0]), float(c[1]),
                                  float(v_shot), float(slide),
                                  float(theta_min), float(tau),
                                  float(robot_radius), float(reach), _ptr(out))
        return dict(zip(("theta", "dir", "t_line", "t_opp", "shoot",
                         "margin"), out.tolist()))

    def shot_gap(self, state: State, c, r):
        start = ctypes.c_double()
        th = self.lib.pps_oracle_shot_gap(state.ref, float(c[0]), float(c[1]),
                                          float(r), ctypes.byref(start))
        return th, start.value

    def dpps_search(self, batch: dict, ndir, npow, params: dict, *,
                    dense=False, n_threads=0):
        """The direction x power search over a batch with teammates."""
        ball = np.asarray(batch["ball"], np.float64)
        S = ball.shape[0]
        sc = np.ascontiguousarray(np.stack(
            [ball[:, 0], ball[:, 1]] + [np.asarray(batch[k], np.float64)
                                        for k in SCALARS[2:]], axis=1))
        J = max(batch["opp_pos"].shape[1], batch["team_pos"].shape[1])

        def robots(pos, vel):
            out = np.zeros((S, J, 4), np.float64)
            n = pos.shape[1]
            out[:, :n, :2] = pos
            out[:, :n, 2:] = vel
            return np.ascontiguousarray(out)

        team = robots(np.asarray(batch["team_pos"], np.float64),
                      np.asarray(batch["team_vel"], np.float64))
        opp = robots(np.asarray(batch["opp_pos"], np.float64),
                     np.asarray(batch["opp_vel"], np.float64))
        n_team = np.ascontiguousarray(np.asarray(
            batch.get("n_team", np.full(S, batch["team_pos"].shape[1])),
            np.int32))
        n_opp = np.ascontiguousarray(np.asarray(batch["n_opp"], np.int32))
        K = np.ascontiguousarray(np.asarray(batch["K"], np.int32))
        prm = np.array([float(params[k]) for k in DPPS_PARAMS], np.float64)
        C = int(ndir) * int(npow)
        out = {"best_idx": np.empty(S, np.int64),
               "best_score": np.empty(S, np.float64),
               "n_feasible": np.empty(S, np.int64)}
        if dense:
            out["feasible"] = np.empty((S, C), np.uint8)
            out["score"] = np.empty((S, C), np.float64)
            out["t_team"] = np.empty((S, C), np.float64)
            out["t_opp"] = np.empty((S, C), np.float64)
        rc = self.lib.pps_oracle_dpps_search(
            S, _ptr(sc), _ptr(n_team), _ptr(team), _ptr(n_opp), _ptr(opp),
            _ptr(K), J, int(ndir), int(npow), _ptr(prm),
            _ptr(out["best_idx"]), _ptr(out["best_score"]),
            _ptr(out["n_feasible"]), _ptr(out.get("feasible")),
            _ptr(out.get("score")), _ptr(out.get("t_team")),
            _ptr(out.get("t_opp")), int(n_threads))
        if rc != 0:
            raise ValueError("oracle rejected the batch")
        return out


    # -- running points (pps_oracle.h, R) --
    def run_point(self, st: DState, params: dict, p):
        """Score, zone, the five criteria and candidacy of point p."""
        prm = np.array([float(params[k]) for k in RUN_PARAMS], np.float64)
        out = np.empty(8, np.float64)
        self.lib.pps_oracle_run_point(st.ref, _ptr(prm), float(p[0]),
                                      float(p[1]), _ptr(out))
        r = {"score": out[0], "zone": int(out[1]), "candidate": bool(out[7])}
        r.update(zip(RUN_CRITERIA, out[2:7].tolist()))
        return r

    def run_zone(self, st: DState, p, params: dict | None = None) -> int:
        """Zone 0..3 of point p, -1 outside the attacking half; the edge
        tolerance comes from params' spacing (default 0.1 m)."""
        params = params or {"spacing": 0.1}
        prm = np.zeros(len(RUN_PARAMS), np.float64)
        prm[0] = float(params["spacing"])
        return self.lib.pps_oracle_run_zone(st.ref, _ptr(prm), float(p[0]),
                                            float(p[1]))

    def run_choose(self, best_idx, best_score, avoid, n_run):
        bi = np.ascontiguousarray(np.asarray(best_idx, np.int64))
        bs = np.ascontiguousarray(np.asarray(best_score, np.float64))
        ch = np.empty(4, np.int32)
        self.lib.pps_oracle_run_choose(_ptr(bi), _ptr(bs), int(avoid),
                                       int(n_run), _ptr(ch))
        return ch

    def run_search(self, batch: dict, params: dict, *, pass_points=None,
                   dense=False, n_threads=0):
        """Running points of every state of a batch (teammates unused).
        pass_points: (S, 2) best passing points, NaN for none."""
        ball = np.asarray(batch["ball"], np.float64)
        S = ball.shape[0]
        sc = np.ascontiguousarray(np.stack(
            [ball[:, 0], ball[:, 1]] + [np.asarray(batch[k], np.float64)
                                        for k in SCALARS[2:]], axis=1))
        J = batch["opp_pos"].shape[1]
        opp = np.zeros((S, J, 4), np.float64)
        opp[:, :, :2] = batch["opp_pos"]
        opp[:, :, 2:] = batch["opp_vel"]
        opp = np.ascontiguousarray(opp)
        n_opp = np.ascontiguousarray(np.asarray(batch["n_opp"], np.int32))
        prm = np.array([float(params[k]) for k in RUN_PARAMS], np.float64)
        pp = None if pass_points is None else np.ascontiguousarray(
            np.asarray(pass_points, np.float64).reshape(S, 2))
        out = {"best_idx": np.empty((S, 4), np.int64),
               "best_score": np.empty((S, 4), np.float64),
               "chosen": np.empty((S, 4), np.int32),
               "avoided": np.empty(S, np.int32)}
        if dense:
            g = prm[0]
            L = float(np.asarray(batch["field_len"]).reshape(-1)[0])
            W = float(np.asarray(batch["field_wid"]).reshape(-1)[0])
            nx, ny = int(round(0.5 * L / g)) + 1, int(round(W / g)) + 1
            out["score"] = np.empty((S, ny, nx), np.float64)
        rc = self.lib.pps_oracle_run_search(
            S, _ptr(sc), _ptr(n_opp), _ptr(opp), J, _ptr(prm), _ptr(pp),
            _ptr(out["best_idx"]), _ptr(out["best_score"]),
            _ptr(out["chosen"]), _ptr(out["avoided"]), _ptr(out.get("score")),
            int(n_threads))
        if rc != 0:
            raise ValueError("oracle rejected the batch")
        return out


class _DState(ctypes.Structure):
    _fields_ = [("sc", ctypes.c_void_p), ("n_team", ctypes.c_int),
                ("team", ctypes.c_void_p), ("n_opp", ctypes.c_int),
                ("opp", ctypes.c_void_p), ("K", ctypes.c_int)]


class DState:
    """One state of the direction x power search (float64 arrays): scalars
    as ``State``, receivers ``team`` and ``opp`` as (n, 4) x, y, vx, vy."""

    def __init__(self, scalars: dict, team, opp, K: int):
        self.sc = np.array([float(scalars[k]) for k in SCALARS], np.float64)
        self.team = np.ascontiguousarray(
            np.asarray(team, np.float64).reshape(-1, 4))
        self.opp = np.ascontiguousarray(
            np.asarray(opp, np.float64).reshape(-1, 4))
        self.K = int(K)
        self._c = _DState(_ptr(self.sc), self.team.shape[0], _ptr(self.team),
                          self.opp.shape[0], _ptr(self.opp), self.K)

    @property
    def ref(self):
        return ctypes.byref(self._c)


def dstate_of(batch: dict, s: int) -> DState:
    """State s of a batch with teammates (team_pos, team_vel)."""
    n = int(batch["n_opp"][s])
    nt = int(batch["n_team"][s]) if "n_team" in batch else \
        batch["team_pos"].shape[1]
    opp = np.concatenate([np.asarray(batch["opp_pos"][s, :n], np.float64),
                          np.asarray(batch["opp_vel"][s, :n], np.float64)],
                         axis=1)
    team = np.concatenate([np.asarray(batch["team_pos"][s, :nt], np.float64),
                           np.asarray(batch["team_vel"][s, :nt], np.float64)],
                          axis=1)
    sc = {"ball_x": batch["ball"][s][0], "ball_y": batch["ball"][s][1]}
    for k in SCALARS[2:]:
        sc[k] = batch[k][s]
    return DState(sc, team, opp, int(batch["K"][s]))


def state_of(batch: dict, s: int) -> State:
    """State ``s`` of a batch, in the oracle's layout."""
    n = int(batch["n_opp"][s])
    opp = np.concatenate([np.asarray(batch["opp_pos"][s, :n], np.float64),
                          np.asarray(batch["opp_vel"][s, :n], np.float64)],
                         axis=1)
    sc = {"ball_x": batch["ball"][s][0], "ball_y": batch["ball"][s][1]}
    for k in SCALARS[2:]:
        sc[k] = batch[k][s]
    return State(sc, opp, int(batch["K"][s]))


def default() -> Oracle:
    """The oracle built from ``pps_oracle.c`` (loaded once)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle()
        return _default


_default = None


def __getattr__(name):
    # Module-level shortcuts: oracle.ball_time(...) == default().ball_time(...)
    if name in ("grid", "ball_time", "intercept_time", "min_intercept",
                "min_intercept_many",
                "margin", "shot_angle", "score", "search", "max_threads",
                "dpps_path", "dpps_group", "dpps_candidate", "dpps_search",
                "pass_power", "shoot", "shot_gap", "run_point", "run_zone",
                "run_choose", "run_search"):
        return getattr(default(), name)
    raise AttributeError(name)
