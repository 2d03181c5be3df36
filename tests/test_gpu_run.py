"""The running-point search (Sec. 5.1-5.2) on the GPU against the FP64
oracle.

Dense scores are compared point by point, except where a decision of the
method sits within rounding of its threshold (the defence area's edge, an
opponent as near the ball as the point); the best point of each zone is
compared through the oracle's score of it, and the zone choice wherever
the zone scores are not within rounding of a tie.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1909_07717_gb300 import pps, synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def searcher():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    s = pps.Searcher(max_states=4096, max_opp=16)
    yield s
    s.close()


def _device(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8)
                            .reshape(-1).copy()).cuda()


def _run(s, batch, prm, dense=True, pass_best=None, stride=None):
    torch = s.torch
    n = batch["ball"].shape[0]
    p = pps.rparams_from_dict(prm)
    states = _device(torch, pps.pack_dstates(batch))
    out = torch.empty(n * pps.RBEST_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    sc = None
    if dense:
        nx, ny = pps.pps_run_grid(float(batch["field_len"][0]),
                                  float(batch["field_wid"][0]), p.spacing)
        stride = stride or nx * ny
        sc = torch.full((n, stride), 7.0, dtype=torch.float32, device="cuda")
    pb = None if pass_best is None else pass_best
    pps.pps_run_points(s.ctx, states.data_ptr(), n, p, out.data_ptr(),
                       pb.data_ptr() if pb is not None else None,
                       sc.data_ptr() if sc is not None else None,
                       stride or 0)
    torch.cuda.synchronize()
    r = np.frombuffer(out.cpu().numpy().tobytes(), pps.RBEST_DTYPE)
    return r, (sc.cpu().numpy() if sc is not None else None)


def _ambiguous(batch, s, nx, ny, prm, eps=1e-5):
    """Grid points where the candidacy, the avoidance flag or the zone is
    within rounding of flipping."""
    g = prm["spacing"]
    L = float(batch["field_len"][s])
    W = float(batch["field_wid"][s])
    x = np.minimum(np.arange(nx) * g, L / 2)
    y = np.minimum(-W / 2 + np.arange(ny) * g, W / 2)
    X, Y = np.meshgrid(x, y)
    b = batch["ball"][s].astype(np.float64)
    n = int(batch["n_opp"][s])
    o = batch["opp_pos"][s, :n].astype(np.float64)
    dmin = np.min(np.hypot(o[:, 0] - b[0], o[:, 1] - b[1])) if n else np.inf
    db = np.hypot(X - b[0], Y - b[1])
    tol = g / 1024
    x0 = L / 2 - prm["def_depth"] + tol
    y1 = prm["def_width"] / 2 - tol
    ys = min(max(b[1], -W / 4), W / 4) - tol
    return ((np.abs(db - dmin) < eps) | (np.abs(X - x0) < eps)
            | (np.abs(np.abs(Y) - y1) < eps) | (np.abs(X - L / 4 + tol) < eps)
            | (np.abs(Y - ys) < eps))


def test_dense_scores_and_zone_bests_match_the_oracle(searcher):
    prm = synth.run_oracle_params()
    batch = synth.run_states(41, 12)
    got, dense = _run(searcher, batch, synth.RUN_PARAMS)
    ref = oracle.run_search(batch, prm, dense=True)
    ny, nx = ref["score"].shape[1:]
    compared = 0
    for s in range(12):
        assert got[s]["status"] == 0
        assert (got[s]["nx"], got[s]["ny"]) == (nx, ny)
        g = dense[s, :nx * ny]
        r = ref["score"][s].reshape(-1)
        amb = _ambiguous(batch, s, nx, ny, prm).reshape(-1)
        ok = ~amb
        assert np.array_equal(np.isinf(g[ok]), np.isinf(r[ok]))
        fin = ok & np.isfinite(r)
        assert np.max(np.abs(g[fin] - r[fin])) <= TOL, s
        compared += int(fin.sum())
        for q in range(4):
            gi = int(got[s]["idx"][q])
            assert gi >= 0 and (np.isfinite(r[gi]) or amb[gi])
            # the GPU's point scores the oracle's best of the zone
            if np.isfinite(r[gi]):
                assert abs(r[gi] - ref["best_score"][s, q]) <= 2 * TOL, (s, q)
            assert abs(got[s]["score"][q] - ref["best_score"][s, q]) <= TOL
            assert got[s]["score"][q] == g[gi]
            j, i = divmod(gi, nx)
            assert got[s]["point"][q][0] == min(np.float32(
                np.float32(i) * np.float32(prm["spacing"])), np.float32(6.0))
            st = oracle.dstate_of(batch, s)
            assert oracle.run_zone(st, got[s]["point"][q], prm) == q or amb[gi]
        # the choice, unless two zone scores tie within rounding
        bs = ref["best_score"][s]
        if abs(bs[2] - bs[3]) > 4 * TOL and abs(bs[0] - bs[1]) > 4 * TOL:
            assert list(got[s]["chosen"]) == list(ref["chosen"][s])
        assert got[s]["avoided"] == -1
    assert compared >= 0.97 * 12 * (nx * ny - 300)


def test_ties_take_the_first_point_of_each_zone(searcher):
    prm = dict(synth.RUN_PARAMS, w_goal=0.0, w_ball=0.0, w_angle=0.0,
               w_guard=0.0, w_avoid=0.0)
    batch = synth.run_states(42, 5)
    got, _ = _run(searcher, batch, prm, dense=False)
    ref = oracle.run_search(batch, synth.run_oracle_params(prm))
    assert np.array_equal(got["idx"], ref["best_idx"].astype(np.int32))
    assert np.all(got["score"] == 0.0)
    assert np.array_equal(got["chosen"], ref["chosen"])


def test_the_best_passing_points_zone_is_avoided(searcher):
    torch = searcher.torch
    batch = synth.run_states(43, 64)
    # the direction x power search over the same states names the pass
    dbatch = synth.dpps_states(43, 64, n_team=6, n_opp=16, K=32)
    for k in ("ball", "opp_pos", "opp_vel", "n_opp"):
        dbatch[k] = batch[k]
    dstates = _device(torch, pps.pack_dstates(dbatch))
    dp = pps.dparams_from_dict(dict(synth.DPPS_PARAMS, n_dir=32, n_pow=16))
    best = torch.empty(64 * pps.DBEST_DTYPE.itemsize, dtype=torch.uint8,
                       device="cuda")
    pps.pps_dpps_search(searcher.ctx, dstates.data_ptr(), 64, dp,
                        best.data_ptr(), None, None)
    torch.cuda.synchronize()
    db = np.frombuffer(best.cpu().numpy().tobytes(), pps.DBEST_DTYPE)
    got, _ = _run(searcher, dbatch, synth.RUN_PARAMS, dense=False,
                  pass_best=best)
    pts = np.where((db["idx"] >= 0)[:, None], db["recv"].astype(np.float64),
                   np.nan)
    ref = oracle.run_search(dbatch, synth.run_oracle_params(),
                            pass_points=pts)
    avoided = 0
    for s in range(64):
        assert got[s]["avoided"] == ref["avoided"][s], s
        avoided += int(ref["avoided"][s] >= 0)
        bs = ref["best_score"][s]
        if abs(bs[2] - bs[3]) > 4 * TOL and abs(bs[0] - bs[1]) > 4 * TOL:
            assert list(got[s]["chosen"]) == list(ref["chosen"][s]), s
        assert got[s]["avoided"] not in [z for z in got[s]["chosen"]
                                         if z >= 0]
    assert avoided >= 10


def test_supporter_counts(searcher):
    batch = synth.run_states(44, 4)
    for n_run in (0, 1, 2, 3):
        got, _ = _run(searcher, batch, dict(synth.RUN_PARAMS, n_run=n_run),
                      dense=False)
        for s in range(4):
            ch = [z for z in got[s]["chosen"] if z >= 0]
            assert len(ch) == n_run
            assert all(z in (2, 3) for z in ch[:2])


def test_full_size_workload(searcher):
    """The benchmark's shape: 12 x 9 m fields, 16 opponents, g = 0.1 m; the
    bookkeeping of every record and four states against the oracle."""
    batch = synth.run_states(synth.RUN_SEED, 1024)
    got, _ = _run(searcher, batch, synth.RUN_PARAMS, dense=False)
    assert np.all(got["status"] == 0)
    assert np.all((got["idx"] >= 0) & (got["idx"] < 61 * 91))
    assert np.all(np.isfinite(got["score"]))
    take = [0, 1, 511, 1023]
    sub = {k: (v[take] if isinstance(v, np.ndarray) else v)
           for k, v in batch.items()}
    ref = oracle.run_search(sub, synth.run_oracle_params(), dense=True)
    for t, s in enumerate(take):
        r = ref["score"][t].reshape(-1)
        for q in range(4):
            gi = int(got[s]["idx"][q])
            assert abs(r[gi] - ref["best_score"][t, q]) <= 2 * TOL


def test_invalid_states_and_arguments(searcher):
    batch = synth.run_states(45, 4)
    batch["n_opp"] = batch["n_opp"].copy()
    batch["n_opp"][1] = 17
    batch["field_len"] = batch["field_len"].copy()
    batch["field_len"][2] = 0.0
    batch["opp_pos"] = batch["opp_pos"].copy()
    batch["opp_pos"][3, 5, 0] = np.nan
    got, dense = _run(searcher, batch, synth.RUN_PARAMS)
    assert got[0]["status"] == 0
    for s in (1, 2, 3):
        assert got[s]["status"] & 1
        assert np.all(got[s]["idx"] == -1) and np.all(got[s]["chosen"] == -1)
    # a score stride too small for the grid
    good = synth.run_states(46, 2)
    got, _ = _run(searcher, good, synth.RUN_PARAMS, stride=100)
    assert np.all(got["status"] & 1)
    # parameters out of range are refused before any launch
    for bad in ({"spacing": 0.0}, {"angle_hi": 0.1}, {"n_run": 5},
                {"guard_cap": float("nan")}):
        with pytest.raises(pps.PpsError):
            _run(searcher, good, dict(synth.RUN_PARAMS, **bad), dense=False)
    # no states: nothing to do
    pps.pps_run_points(searcher.ctx, 0, 0, None, 0)


def test_small_field_fine_grid_and_ragged_opponents(searcher):
    """9 x 6 m fields at 0.05 m (91 x 121 points), 0-16 opponents (a state
    with none has no guard and nothing to avoid): each zone's best against
    the oracle's dense scores."""
    rng = np.random.default_rng(47)
    batch = synth.ssl_states(47, 10, field_len=9.0, field_wid=6.0, n_opp=16,
                             n_team=0, K=1)
    batch["n_opp"] = rng.integers(0, 17, 10).astype(np.int32)
    batch["n_opp"][0] = 0
    batch["opp_pos"][1, 0] = (4.0, 0.3)           # a guard
    prm = dict(synth.RUN_PARAMS, spacing=0.05)
    got, dense = _run(searcher, batch, prm)
    oprm = synth.run_oracle_params(prm)
    ref = oracle.run_search(batch, oprm, dense=True)
    ny, nx = ref["score"].shape[1:]
    assert (nx, ny) == (91, 121)
    for s in range(10):
        assert got[s]["status"] == 0 and (got[s]["nx"], got[s]["ny"]) == (nx, ny)
        r = ref["score"][s].reshape(-1)
        g = dense[s, :nx * ny]
        amb = _ambiguous(batch, s, nx, ny, oprm).reshape(-1)
        fin = ~amb & np.isfinite(r)
        assert np.max(np.abs(g[fin] - r[fin])) <= TOL, s
        for q in range(4):
            gi = int(got[s]["idx"][q])
            assert gi >= 0
            if np.isfinite(r[gi]):
                assert abs(r[gi] - ref["best_score"][s, q]) <= 2 * TOL, (s, q)
    # no opponent: nothing to avoid and no guard, so those criteria are
    # constant and every score is below the sum of the weights
    assert np.all(dense[0, :nx * ny][np.isfinite(dense[0, :nx * ny])] <= 4.0)


def test_other_weights_band_and_area(searcher):
    """Other criterion weights, an angle band from 0, a smaller defence area
    and two supporters: dense scores and zone bests against the oracle."""
    prm = dict(synth.RUN_PARAMS, w_goal=2.0, w_ball=0.5, w_angle=1.5,
               w_guard=0.7, w_avoid=3.0, ball_ref=1.5, angle_lo=0.0,
               angle_hi=0.4, angle_span=0.8, def_depth=1.0, def_width=2.0,
               guard_cap=1.5, n_run=2)
    batch = synth.run_states(48, 6, def_depth=1.0, def_width=2.0)
    oprm = synth.run_oracle_params(prm)
    got, dense = _run(searcher, batch, prm)
    ref = oracle.run_search(batch, oprm, dense=True)
    ny, nx = ref["score"].shape[1:]
    for s in range(6):
        r = ref["score"][s].reshape(-1)
        g = dense[s, :nx * ny]
        amb = _ambiguous(batch, s, nx, ny, oprm).reshape(-1)
        fin = ~amb & np.isfinite(r)
        assert np.max(np.abs(g[fin] - r[fin])) <= 2 * TOL, s
        for q in range(4):
            gi = int(got[s]["idx"][q])
            if np.isfinite(r[gi]):
                assert abs(r[gi] - ref["best_score"][s, q]) <= 4 * TOL, (s, q)
        assert sum(z >= 0 for z in got[s]["chosen"]) == 2
