"""Shared machinery of the GPU-vs-oracle parity tests.

Tolerances (FP32 GPU against the FP64 oracle on identical FP32 inputs):
  * feasibility mask: identical wherever the oracle margin is more than
    1e-3 s from tau_safe, the ball's reach is not within 1e-4 v^2 of the
    pass length (|v^2 - 2 a D| > 1e-4 v^2), and the pass length is not
    within 1e-5 m of min_pass_dist;
  * intercept times T_k: |dT| <= 1e-5 s + 2 * cond_k, where
    cond_k = |grad_p T_k| * 2e-6 m is how far T_k moves when the sample
    point moves by the rounding of FP32 coordinates on a 12 m field;
    well-conditioned samples (|grad_p T_k| <= 2 s/m: the allowance would be
    at most 8e-6 s) are held to the plain 1e-5 s, and at most 5 % of a
    state's samples (of states with at least 1000) may be outside that
    class (a sample within a metre or two of an opponent moving across the
    line, where the intercept time changes fast with the point; 0.3-3.2 %
    of the samples of the dense parity cases);
  * margins (reachable passes outside the reach band):
    |dm| <= 1e-5 s + 2 * max_k (cond_k + bcond_k), where bcond_k is the
    first-order change of the ball time t(s_k) when v^2 and s_k carry FP32
    rounding: eps (v^2 + 2 a s_k) / (2 a sqrt(v^2 - 2 a s_k)), eps = 2^-24
    (the ball time's slope grows without bound as the ball nears its stop);
  * best score: |ds| <= 1e-5 * max(1, |s|), and the GPU's best candidate
    must be one the oracle scores within that tolerance of its own best.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1909_07717_gb300 import pps

DELTA_P = 2e-6      # m, FP32 position rounding scale on a 12 m field
TOL_T = 1e-5        # s
TOL_MASK = 1e-3     # s
TOL_REACH = 1e-4    # relative to v^2
TOL_SCORE = 1e-5    # relative, floor 1
WELLCOND_GRAD = 2.0       # s/m: samples held to the plain TOL_T
MAX_ILLCOND_FRAC = 0.05   # most samples of a state outside that class


def grid_spec(grid):
    """The oracle's view of a library grid: (g, nx, ny, x0, y0) in FP64."""
    return (float(np.float32(grid.spacing)), grid.nx, grid.ny,
            float(np.float32(grid.x0)), float(np.float32(grid.y0)))


def unpack_mask(words, n_states, V, P):
    w = np.asarray(words).view(np.uint32).reshape(n_states, V, -1)
    bits = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :P].astype(bool), bits[..., P:]


def run_gpu(searcher, batch, grid, speeds, params, debug=True, T=True,
            host=False):
    """Run the library on a batch; returns numpy arrays."""
    import torch
    S = batch["ball"].shape[0]
    V = len(speeds)
    P = grid.nx * grid.ny
    if host:
        rec = pps.pack_states(batch)
        best = np.zeros(S, pps.BEST_DTYPE)
        mask = np.zeros(S * pps.pps_mask_words(grid, V), np.uint32)
        searcher.search_host(rec, grid, speeds, params, best, mask)
        searcher.sync()
        return {"best": best, "mask": mask}
    st = searcher.states_to_device(batch)
    Tstride = int(np.max(batch["K"])) if T else 0
    out = searcher.search(st, S, grid, speeds, params, debug=debug,
                          T_stride=Tstride)
    torch.cuda.synchronize()
    res = {"best": pps.unpack_best(out["best"].cpu().numpy()),
           "mask": out["mask"].cpu().numpy().view(np.uint32)}
    for k in ("margin", "score", "T"):
        if k in out:
            res[k] = out[k].cpu().numpy()
    return res


def sample_points(state: oracle.State, grid, K):
    """FP64 sample positions (P, K, 2) of every pass of a state."""
    g, nx, ny, x0, y0 = grid_spec(grid)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    cx = (x0 + ix * g).reshape(-1)
    cy = (y0 + iy * g).reshape(-1)
    bx, by = state.sc[0], state.sc[1]
    f = np.arange(1, K + 1) / K
    px = bx + f[None, :] * (cx[:, None] - bx)
    py = by + f[None, :] * (cy[:, None] - by)
    return np.stack([px, py], axis=-1), cx, cy


def T_condition(state: oracle.State, grid, K, reach=0.0, h=1e-7):
    """cond[p, k] = |grad T_k| * DELTA_P by central differences of the
    oracle's minimum intercept time around each sample point."""
    pts, _, _ = sample_points(state, grid, K)
    P = pts.shape[0]
    flat = pts.reshape(-1, 2)
    grads = []
    for e in ((h, 0.0), (0.0, h)):
        e = np.array(e)
        tp = oracle.min_intercept_many(state, flat + e, reach)
        tm = oracle.min_intercept_many(state, flat - e, reach)
        with np.errstate(invalid="ignore"):
            grads.append(np.where(np.isfinite(tp) & np.isfinite(tm),
                                  (tp - tm) / (2 * h), 0.0))
    gn = np.hypot(grads[0], grads[1]).reshape(P, K)
    return gn * DELTA_P


def ball_condition(sp, a, D, K):
    """max_k of the FP32 input-rounding sensitivity of the ball time along
    each pass: shape (V, P)."""
    eps = 2.0 ** -24
    f = np.arange(1, K + 1) / K
    s_k = f[None, None, :] * D[None, :, None]
    v2 = (np.asarray(sp, np.float64) ** 2)[:, None, None]
    x = v2 - 2 * a * s_k
    with np.errstate(divide="ignore", invalid="ignore"):
        c = eps * (v2 + 2 * a * s_k) / (2 * a * np.sqrt(np.maximum(x, 0)))
    return np.nan_to_num(c, nan=np.inf, posinf=np.inf).max(axis=2)


def check_state_dense(gpu, orc, batch, s, grid, speeds, params, Tcond=None):
    """Dense comparison of one state; returns a dict of statistics."""
    st = oracle.state_of(batch, s)
    K = st.K
    V = len(speeds)
    g, nx, ny, x0, y0 = grid_spec(grid)
    P = nx * ny
    stats = {}
    mask, pad = unpack_mask(gpu["mask"], batch["ball"].shape[0], V, P)
    assert not pad[s].any(), "mask bits beyond P must be zero"
    feas_o = orc["feasible"][s].astype(bool)
    m_o = orc["margin"][s]
    if Tcond is None:
        Tcond = T_condition(st, grid, K, params.get("reach_radius", 0.0))
    # ---- T_k
    if "T" in gpu:
        To = orc["T"][s, :, :K]
        Tg = gpu["T"][s, :, :K].astype(np.float64)
        both_inf = np.isinf(To) & np.isinf(Tg)
        with np.errstate(invalid="ignore"):   # inf - inf where both are inf
            err = np.where(both_inf, 0.0, np.abs(Tg - To))
        tol = TOL_T + 2 * Tcond
        bad = err > tol
        # well-conditioned: |grad T| <= WELLCOND_GRAD (a sample away from
        # any opponent moving across the line that could reach it first)
        wc = Tcond <= WELLCOND_GRAD * DELTA_P
        stats["T_max_err_wellcond"] = float(err[wc].max(initial=0))
        stats["T_max_err"] = float(err.max(initial=0))
        stats["T_frac_wellcond"] = float(np.mean(wc))
        assert not bad.any(), (
            f"state {s}: {bad.sum()} T_k outside tolerance, worst "
            f"{err[bad].max():.3g} s at cond {Tcond[bad][np.argmax(err[bad])]:.3g}")
        assert stats["T_max_err_wellcond"] <= TOL_T, (
            f"state {s}: well-conditioned T_k off by "
            f"{stats['T_max_err_wellcond']:.3g} s")
        # (a share is only meaningful over many samples: tiny grids aside)
        assert wc.size < 1000 or \
            1.0 - stats["T_frac_wellcond"] <= MAX_ILLCOND_FRAC, (
                f"state {s}: {1 - stats['T_frac_wellcond']:.3f} of the "
                f"samples need the conditioning allowance")
    # ---- bands
    _, cx, cy = sample_points(st, grid, 1)
    D = np.hypot(cx - st.sc[0], cy - st.sc[1])
    a = st.sc[2]
    sp = np.asarray(speeds, np.float64)
    reach_gap = np.abs(sp[:, None] ** 2 - 2 * a * D[None, :]) / sp[:, None] ** 2
    in_band = ((np.abs(m_o - params["tau_safe"]) <= TOL_MASK)
               | (reach_gap <= TOL_REACH)
               | (np.abs(D - params["min_pass_dist"]) <= 1e-5)[None, :])
    stats["mask_band_frac"] = float(in_band.mean())
    stats["mask_band_count"] = int(in_band.sum())
    diff = (mask[s] != feas_o) & ~in_band
    assert not diff.any(), f"state {s}: {diff.sum()} mask bits differ"
    # ---- margins
    tolm = 0.0
    if "margin" in gpu:
        mg = gpu["margin"][s].astype(np.float64)
        reach_o = np.isfinite(m_o) | (m_o == np.inf)
        neg = ~(reach_gap > TOL_REACH)
        cmp = reach_o & ~neg & np.isfinite(m_o)
        tolm = TOL_T + 2 * (Tcond.max(axis=1)[None, :]
                            + ball_condition(sp, a, D, K))
        with np.errstate(invalid="ignore"):   # equal infinities: nan, masked below
            err = np.abs(mg - m_o)
        bad = cmp & (err > tolm)
        stats["margin_max_err"] = float(err[cmp].max(initial=0))
        assert not bad.any(), (
            f"state {s}: {bad.sum()} margins outside tolerance, worst "
            f"{err[bad].max():.3g}")
        # infinities agree (no opponents: +inf; ball stops short: -inf)
        clear = reach_gap > TOL_REACH
        assert np.array_equal(np.isposinf(mg)[clear], np.isposinf(m_o)[clear])
        assert np.array_equal(np.isneginf(mg)[clear], np.isneginf(m_o)[clear])
    # ---- scores of candidates feasible on both sides
    if "score" in gpu:
        sg = gpu["score"][s].astype(np.float64)
        so = orc["score"][s]
        both = mask[s] & feas_o
        tols = (TOL_SCORE * np.maximum(1, np.abs(so))
                + params["w_margin"] * np.where(
                    m_o < params["margin_cap"] + 1e-4, tolm, 0))
        with np.errstate(invalid="ignore"):   # equal infinities: nan, masked below
            err = np.abs(sg - so)
        stats["score_max_err"] = float(err[both].max(initial=0))
        bad = both & (err > tols)
        assert not bad.any(), f"state {s}: {bad.sum()} scores differ"
        assert np.all(np.isneginf(sg[~mask[s]]))
    return stats


def check_best(gpu, orc, s, nx, P, dense=True):
    """The GPU's best pass against the oracle's."""
    b = gpu["best"][s]
    assert b["status"] == 0, f"state {s}: status {b['status']}"
    ob, os_ = int(orc["best_idx"][s]), float(orc["best_score"][s])
    if ob < 0:
        assert b["idx"] == -1 or dense, f"state {s}: GPU found a pass"
        if b["idx"] == -1:
            return
    if b["idx"] < 0:
        raise AssertionError(f"state {s}: GPU found no pass, oracle {ob}")
    tol = TOL_SCORE * max(1.0, abs(os_))
    assert abs(float(b["score"]) - os_) <= tol, (
        f"state {s}: best score {b['score']} vs oracle {os_}")
    if dense:
        so = orc["score"][s].reshape(-1)
        assert so[b["idx"]] >= os_ - tol, (
            f"state {s}: GPU best idx {b['idx']} scores {so[b['idx']]} in "
            f"the oracle, best {os_}")
    v, p = divmod(int(b["idx"]), P)
    assert v == b["speed_idx"] and p == b["iy"] * nx + b["ix"]


def check_mask_one(bits, orc_feasible, orc_margin, state, gspec, speeds,
                   params):
    """Mask bits (V, P) of one state against the oracle outside the bands;
    returns the number of in-band candidates."""
    g, nx, ny, x0, y0 = gspec
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    cx = (x0 + ix * g).reshape(-1)
    cy = (y0 + iy * g).reshape(-1)
    D = np.hypot(cx - state.sc[0], cy - state.sc[1])
    sp = np.asarray(speeds, np.float64)
    gap = np.abs(sp[:, None] ** 2 - 2 * state.sc[2] * D[None, :]) / \
        sp[:, None] ** 2
    band = ((np.abs(orc_margin - params["tau_safe"]) <= TOL_MASK)
            | (gap <= TOL_REACH)
            | (np.abs(D - params["min_pass_dist"]) <= 1e-5)[None, :])
    diff = (bits != orc_feasible.astype(bool)) & ~band
    assert not diff.any(), f"{diff.sum()} mask bits differ outside the bands"
    return int(band.sum())


def words_to_bits(words, V, P):
    w = np.asarray(words).view(np.uint32).reshape(V, -1)
    bits = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    assert not bits[:, P:].any(), "mask bits beyond P must be zero"
    return bits[:, :P].astype(bool)
