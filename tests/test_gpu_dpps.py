"""The direction x power search (the paper's own parameterisation,
Sec. 4.2) on the GPU against the FP64 oracle.

Every candidate's teammate and opponent interception times, feasibility
and score are compared wherever the oracle's sampled decisions are not
within 0.1 ms of flipping (FP32 and FP64 may take such a decision
differently, and then the first interception moves by a sample) and the
ball is not in its ill-conditioned last crawl before the stop; the times
within a bound derived from their float32 roundings, the score within
1e-5 relative plus those times' bounds; the best candidate is compared
through the oracle's score of it.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1909_07717_gb300 import pps, synth

pytestmark = pytest.mark.gpu
EPS = 1e-4          # s: a sampled decision this close to flipping is skipped
TOL_T = 1e-5        # s: intercept times
TOL_SCORE = 1e-5    # relative, floor 1
ROUNDINGS = 16      # float32 roundings in the inputs of a ball time
STOP_BAND = 1e-2    # remaining ball speed / v below which a ball time is
                    # ill-conditioned (as the receive-point parity)


@pytest.fixture(scope="module")
def searcher():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    s = pps.Searcher(max_states=1024, max_opp=16)
    yield s
    s.close()


def _run(s, batch, prm, dbg=True):
    torch = s.torch
    n = batch["ball"].shape[0]
    p = pps.dparams_from_dict(prm)
    rec = torch.from_numpy(pps.pack_dstates(batch).view(np.uint8).copy()).cuda()
    best = torch.empty(n * 48, dtype=torch.uint8, device="cuda")
    words = pps.pps_dpps_mask_words(p)
    mask = torch.full((n, words), -1, dtype=torch.int32, device="cuda")
    C = p.n_dir * p.n_pow
    d = torch.empty((n, C, 3), dtype=torch.float32, device="cuda") if dbg else None
    pps.pps_dpps_search(s.ctx, rec.data_ptr(), n, p, best.data_ptr(),
                        mask.data_ptr(), d.data_ptr() if dbg else None)
    torch.cuda.synchronize()
    b = np.frombuffer(best.cpu().numpy().tobytes(), pps.DBEST_DTYPE)
    m = mask.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(m.view(np.uint8), axis=1, bitorder="little")[:, :C]
    return b, bits, (d.cpu().numpy() if dbg else None)


def _oracle_candidates(batch, prm, s):
    st = oracle.dstate_of(batch, s)
    op = synth.dpps_oracle_params(prm)
    return [[oracle.dpps_candidate(st, op, prm["n_dir"], prm["n_pow"], i, j)
             for j in range(prm["n_pow"])] for i in range(prm["n_dir"])]


def _rolling_speed(prm, j):
    v0 = prm["v_lo"] + j * (prm["v_hi"] - prm["v_lo"]) / (prm["n_pow"] - 1)
    return prm["slide"] * v0


def time_tolerance(t, v, a):
    """Bound on the FP32 error of a first-interception time t of a ball
    rolling from v with deceleration a, or None inside the ill-conditioned
    band.  A ball time t = 2 s / (v + r), r = sqrt(v^2 - 2 a s) = v - a t,
    moves by (ds + t dv) / r when s and v move by ds and dv; both carry
    the float32 rounding of a few operations (ROUNDINGS x 2^-24 of s and of
    v), so |dt| <= ROUNDINGS 2^-24 (s + v t) / r, plus TOL_T for the
    intercept time the decision compares it with.  At the stop
    (t >= v / a: the ball at rest, or a robot arriving after it stopped)
    the time is v / a or the robot's intercept time: TOL_T plus the
    rounding of t.  A ball still moving slower than STOP_BAND v is
    ill-conditioned (r -> 0)."""
    if math.isinf(t):
        return 0.0
    r = v - a * t
    eps = ROUNDINGS * 2.0 ** -24
    if r <= 1e-9 * v:
        return TOL_T + eps * t
    if r < STOP_BAND * v:
        return None
    s = v * t - 0.5 * a * t * t
    return TOL_T + eps * (s + v * t) / r


DIR_TOL = 2e-5      # rad: the shot direction (asserted below)


def line_time_tolerance(t, v, a, direction):
    """time_tolerance of a time along a shot, plus the shift of the shot's
    path: a direction off by DIR_TOL moves the distance s to a point at a
    fixed x (the goal line) by s |tan(dir)| DIR_TOL, and the time by that
    over the ball's speed there."""
    base = time_tolerance(t, v, a)
    if base is None or math.isinf(t):
        return base
    r = max(v - a * t, 1e-9 * v)
    s = v * t - 0.5 * a * t * t
    return base + s * abs(math.tan(direction)) * DIR_TOL / r


def score_tolerance(c, prm, j, a_ball):
    """Bound on the FP32 error of a feasible candidate's score: 1e-5
    relative (floor 1) plus its two times' bounds weighted as the score
    weighs them (w_time t_team, w_delta (t_opp - t_team)); None when a time
    is in the ill-conditioned band."""
    v = _rolling_speed(prm, j)
    tt = time_tolerance(c["t_team"], v, a_ball)
    to = time_tolerance(c["t_opp"], v, a_ball)
    if tt is None or to is None:
        return None
    return (TOL_SCORE * max(1.0, abs(c["score"]))
            + (prm["w_time"] + prm["w_delta"]) * tt + prm["w_delta"] * to)


def _close(a, b, tol):
    if math.isinf(a) or math.isinf(b):
        return math.isinf(a) and math.isinf(b)
    return abs(a - b) <= tol


def _compare_candidates(batch, prm, best, bits, dbg):
    """Every candidate of every state against the oracle; returns the
    number of candidates skipped (decision within EPS of flipping, or a
    time in the ill-conditioned band), the number compared, and the largest
    score error as a share of its tolerance."""
    n_pow = prm["n_pow"]
    excluded = total = 0
    worst = 0.0
    for s in range(batch["ball"].shape[0]):
        ref = _oracle_candidates(batch, prm, s)
        a_ball = float(batch["ball_decel"][s])
        for i in range(prm["n_dir"]):
            for j in range(n_pow):
                c = ref[i][j]
                idx = i * n_pow + j
                g_tt, g_to, g_sc = dbg[s, idx]
                total += 1
                # the mask and the debug output agree everywhere
                assert bits[s, idx] == (g_sc > -np.inf)
                v = _rolling_speed(prm, j)
                if c["m_team"] <= EPS:
                    excluded += 1
                    continue
                tt = time_tolerance(c["t_team"], v, a_ball)
                if tt is None:
                    excluded += 1
                    continue
                assert _close(g_tt, c["t_team"], tt), (s, i, j, g_tt, c)
                if math.isinf(c["t_team"]):
                    assert bits[s, idx] == 0
                    continue
                if c["m_opp"] <= EPS:
                    excluded += 1
                    continue
                to = time_tolerance(c["t_opp"], v, a_ball)
                if to is None:
                    excluded += 1
                    continue
                assert _close(g_to, c["t_opp"], to), (s, i, j, g_to, c)
                gap = c["t_opp"] - c["t_team"] - prm["tau_delta"]
                # an exact tie (both teams get the ball at rest, at v / a,
                # and tau = 0) is decided the same way on both sides
                if gap != 0.0 and abs(gap) <= EPS:
                    excluded += 1
                    continue
                assert bits[s, idx] == int(c["feasible"]), (s, i, j)
                if c["feasible"]:
                    tol = score_tolerance(c, prm, j, a_ball)
                    err = abs(g_sc - c["score"])
                    worst = max(worst, err / tol)
                    assert err <= tol, (s, i, j, g_sc, c, tol)
        # the best: its oracle score is the oracle's best
        fe = [(c["score"], i * n_pow + j) for i in range(prm["n_dir"])
              for j, c in enumerate(ref[i]) if c["feasible"]]
        b = best[s]
        assert b["status"] == 0
        if not fe:
            assert b["idx"] == -1
            continue
        ob, oi = max(fe)
        gi = int(b["idx"])
        assert gi >= 0 and bits[s, gi] == 1
        gc = ref[gi // n_pow][gi % n_pow]
        oc = ref[oi // n_pow][oi % n_pow]
        tg = score_tolerance(gc, prm, gi % n_pow, a_ball)
        to_ = score_tolerance(oc, prm, oi % n_pow, a_ball)
        assert tg is not None and to_ is not None, (gc, oc)
        assert gc["feasible"] and abs(gc["score"] - ob) <= tg + to_, (gc, ob)
        assert abs(float(b["score"]) - gc["score"]) <= tg
        assert b["n_feasible"] == bits[s].sum()
        assert b["dir"] == gi // n_pow and b["pow"] == gi % n_pow
    return excluded, total, worst


@pytest.mark.parametrize("n_pow", [32, 24])
def test_candidates_match_the_oracle(searcher, n_pow):
    """Every candidate's teammate and opponent times within time_tolerance,
    its feasibility exact and its score within 1e-5 relative plus the
    times' tolerances (weighted as the score weighs them), except where a
    sampled decision is within EPS of flipping or a time falls in the
    ill-conditioned band -- at most 1 % of the candidates, counted."""
    prm = dict(synth.DPPS_PARAMS, n_dir=32, n_pow=n_pow)
    batch = synth.dpps_states(31, 4, n_team=6, n_opp=7, K=32)
    best, bits, dbg = _run(searcher, batch, prm)
    excluded, total, worst = _compare_candidates(batch, prm, best, bits, dbg)
    print(f"excluded {excluded} of {total} candidates; largest score error "
          f"/ tolerance {worst:.3f}")
    assert excluded <= 0.01 * total, (excluded, total)


def test_full_size_states_against_the_oracle(searcher):
    """The benchmark's shape (16 v 16, 128 x 64 over 1..6.5 m/s, K = 64) on
    64 states: every record's bookkeeping, and the best of four states
    against the oracle's full search."""
    prm = dict(synth.DPPS_PARAMS)
    batch = synth.dpps_states(synth.DPPS_SEED, 64)
    best, bits, _ = _run(searcher, batch, prm, dbg=False)
    assert np.all(best["status"] == 0)
    assert np.array_equal(best["n_feasible"], bits.sum(axis=1))
    has = best["idx"] >= 0
    assert np.all(bits[has, best["idx"][has]] == 1)
    take = [0, 1, 2, 3]
    sub = {k: (v[take] if isinstance(v, np.ndarray) else v)
           for k, v in batch.items()}
    ref = oracle.dpps_search(sub, prm["n_dir"], prm["n_pow"],
                             synth.dpps_oracle_params(prm))
    for t, s in enumerate(take):
        if ref["best_idx"][t] < 0:
            assert best[s]["idx"] == -1
            continue
        st = oracle.dstate_of(batch, s)
        gi = int(best[s]["idx"])
        gc = oracle.dpps_candidate(st, synth.dpps_oracle_params(prm),
                                   prm["n_dir"], prm["n_pow"],
                                   gi // prm["n_pow"], gi % prm["n_pow"])
        oi = int(ref["best_idx"][t])
        oc = oracle.dpps_candidate(st, synth.dpps_oracle_params(prm),
                                   prm["n_dir"], prm["n_pow"],
                                   oi // prm["n_pow"], oi % prm["n_pow"])
        a_ball = float(batch["ball_decel"][s])
        tg = score_tolerance(gc, prm, gi % prm["n_pow"], a_ball)
        to_ = score_tolerance(oc, prm, oi % prm["n_pow"], a_ball)
        assert gc["feasible"] and tg is not None and to_ is not None
        assert abs(gc["score"] - ref["best_score"][t]) <= tg + to_
        assert abs(float(best[s]["score"]) - gc["score"]) <= tg


def test_large_and_small_work_items_agree(searcher):
    """1024 states at the benchmark's shape: the search cuts the first
    states into work items of 1024 candidates and the last ones into items
    of 256.  Every state's record and mask bits must not depend on which:
    the first 64 and the last 64 states, searched again as batches of their
    own (small items only), give the same bytes."""
    prm = dict(synth.DPPS_PARAMS)
    batch = synth.dpps_states(synth.DPPS_SEED + 1, 1024)
    best, bits, _ = _run(searcher, batch, prm, dbg=False)
    assert np.all(best["status"] == 0)
    assert np.array_equal(best["n_feasible"], bits.sum(axis=1))
    for sl in (slice(0, 64), slice(960, 1024)):
        sub = {k: (v[sl] if isinstance(v, np.ndarray) else v)
               for k, v in batch.items()}
        b2, bits2, _ = _run(searcher, sub, prm, dbg=False)
        assert b2.tobytes() == best[sl].tobytes()
        assert np.array_equal(bits2, bits[sl])


def test_invalid_states_and_empty_teams(searcher):
    prm = dict(synth.DPPS_PARAMS, n_dir=16, n_pow=32)
    batch = synth.dpps_states(32, 3, n_team=4, n_opp=4, K=16)
    batch["K"] = batch["K"].copy()
    batch["K"][1] = 0
    batch["n_team"] = batch["n_team"].copy()
    batch["n_team"][2] = 0
    best, bits, _ = _run(searcher, batch, prm, dbg=False)
    assert best[1]["idx"] == -2 and best[1]["status"] & 1
    assert best[2]["idx"] == -1 and bits[2].sum() == 0
    assert best[0]["status"] == 0


def _device(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8)
                            .reshape(-1).copy()).cuda()


def test_pass_powers_match_the_oracle(searcher):
    torch = searcher.torch
    batch = synth.dpps_states(33, 6, n_team=5, n_opp=5, K=32)
    rng = np.random.default_rng(4)
    q = np.zeros(120, pps.PASS_QUERY_DTYPE)
    q["state"] = rng.integers(0, 6, 120)
    q["receiver"] = rng.integers(0, 5, 120)
    q["target"] = rng.uniform([-6, -4.5], [6, 4.5], (120, 2))
    q["receiver"][0] = 7          # no such receiver
    q["state"][1] = 9             # no such state
    states = _device(torch, pps.pack_dstates(batch))
    qd = _device(torch, q)
    out = torch.empty(120 * pps.PASS_POWER_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    p = pps.dparams_from_dict(synth.DPPS_PARAMS)
    pps.pps_pass_powers(searcher.ctx, states.data_ptr(), 6, qd.data_ptr(),
                        120, 0.3, p, out.data_ptr())
    torch.cuda.synchronize()
    g = np.frombuffer(out.cpu().numpy().tobytes(), pps.PASS_POWER_DTYPE)
    assert g["status"][0] == 1 and g["status"][1] == 1
    assert np.isnan(g["v0"][0])
    for i in range(2, 120):
        st = oracle.dstate_of(batch, int(q["state"][i]))
        r = oracle.pass_power(st, int(q["receiver"][i]), q["target"][i],
                              buffer=0.3)
        assert g["status"][i] == 0
        assert abs(g["t_recv"][i] - r["t_recv"]) <= 1e-5 * (1 + r["t_recv"])
        assert abs(g["v1"][i] - r["v1"]) <= 1e-5 * (1 + r["v1"])
        if abs(r["v0"] - 6.5) > 1e-4 and abs(r["v0"] - 1.0) > 1e-4:
            assert g["clamped"][i] == r["clamped"]
        assert abs(g["v0"][i] - r["v0"]) <= 1e-5 * (1 + r["v0"])


def test_shooting_decisions_match_the_oracle(searcher):
    torch = searcher.torch
    batch = synth.dpps_states(34, 6, n_team=4, n_opp=8, K=32)
    rng = np.random.default_rng(5)
    n = 200
    q = np.zeros(n, pps.SHOT_QUERY_DTYPE)
    q["state"] = rng.integers(0, 6, n)
    q["from"] = rng.uniform([-2, -4], [6, 4], (n, 2))
    states = _device(torch, pps.pack_dstates(batch))
    qd = _device(torch, q)
    out = torch.empty(n * pps.SHOT_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    p = pps.dparams_from_dict(synth.DPPS_PARAMS)
    pps.pps_shoot(searcher.ctx, states.data_ptr(), 6, qd.data_ptr(), n, 5.0,
                  0.1, p, out.data_ptr())
    torch.cuda.synchronize()
    g = np.frombuffer(out.cpu().numpy().tobytes(), pps.SHOT_DTYPE)
    shots = checked = 0
    v = synth.DPPS_PARAMS["slide"] * 5.0
    for i in range(n):
        st = oracle.dstate_of(batch, int(q["state"][i]))
        a_ball = float(batch["ball_decel"][int(q["state"][i])])
        r = oracle.shoot(st, q["from"][i], v_shot=5.0, theta_min=0.1)
        assert g["status"][i] == 0
        assert abs(g["theta"][i] - r["theta"]) <= 2e-5
        if r["theta"] > 0:
            assert abs(g["dir"][i] - r["dir"]) <= DIR_TOL
        tl = line_time_tolerance(r["t_line"], v, a_ball, r["dir"])
        if tl is None:
            continue
        assert _close(g["t_line"][i], r["t_line"], tl), (i, g[i], r, tl)
        if r["margin"] <= EPS or abs(r["theta"] - 0.1) <= 1e-5:
            continue
        to = line_time_tolerance(r["t_opp"], v, a_ball, r["dir"])
        if to is None:
            continue
        assert _close(g["t_opp"][i], r["t_opp"], to), (i, g[i], r, to)
        if math.isfinite(r["t_opp"]) and abs(r["t_opp"] - r["t_line"]) <= EPS:
            continue
        assert g["shoot"][i] == r["shoot"], (i, g[i], r)
        shots += int(r["shoot"])
        checked += 1
    assert checked >= 0.9 * n and 0 < shots < checked


@pytest.mark.parametrize("over", [
    dict(tau_delta=0.1, reach_radius=0.05),        # threshold, general path
    dict(slide=1.0, delta_cap=0.5, w_refr=2.0, w_dist=0.5, v_lo=2.0,
         v_hi=5.0),
])
def test_candidates_match_the_oracle_with_other_parameters(searcher, over):
    prm = dict(synth.DPPS_PARAMS, n_dir=16, n_pow=32, **over)
    batch = synth.dpps_states(35, 3, n_team=5, n_opp=6, K=24)
    best, bits, dbg = _run(searcher, batch, prm)
    excluded, total, worst = _compare_candidates(batch, prm, best, bits, dbg)
    print(f"excluded {excluded} of {total} candidates; largest score error "
          f"/ tolerance {worst:.3f}")
    assert excluded <= 0.01 * total, (excluded, total)


def test_pass_powers_with_other_limits(searcher):
    """No buffer, no slide and a narrower kick range (more clamping)."""
    torch = searcher.torch
    batch = synth.dpps_states(36, 4, n_team=4, n_opp=4, K=16)
    rng = np.random.default_rng(6)
    q = np.zeros(80, pps.PASS_QUERY_DTYPE)
    q["state"] = rng.integers(0, 4, 80)
    q["receiver"] = rng.integers(0, 4, 80)
    q["target"] = rng.uniform([-6, -4.5], [6, 4.5], (80, 2))
    states = _device(torch, pps.pack_dstates(batch))
    qd = _device(torch, q)
    out = torch.empty(80 * pps.PASS_POWER_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    p = pps.dparams_from_dict(dict(synth.DPPS_PARAMS, slide=1.0, v_lo=2.0,
                                   v_hi=5.0))
    pps.pps_pass_powers(searcher.ctx, states.data_ptr(), 4, qd.data_ptr(), 80,
                        0.0, p, out.data_ptr())
    torch.cuda.synchronize()
    g = np.frombuffer(out.cpu().numpy().tobytes(), pps.PASS_POWER_DTYPE)
    clamped = 0
    for i in range(80):
        st = oracle.dstate_of(batch, int(q["state"][i]))
        r = oracle.pass_power(st, int(q["receiver"][i]), q["target"][i],
                              buffer=0.0, slide=1.0, v_lo=2.0, v_hi=5.0)
        assert g["status"][i] == 0
        assert abs(g["v1"][i] - r["v1"]) <= 1e-5 * (1 + r["v1"])
        assert abs(g["v0"][i] - r["v0"]) <= 1e-5 * (1 + r["v0"])
        if abs(r["v0"] - 5.0) > 1e-4 and abs(r["v0"] - 2.0) > 1e-4:
            assert g["clamped"][i] == r["clamped"]
        clamped += int(r["clamped"])
    assert clamped > 0
