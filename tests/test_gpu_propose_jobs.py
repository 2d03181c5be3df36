"""The proposal path for states with their own fields and grids
(pps_propose_jobs): the map's cell lattice, off-grid cells ranked last,
the refinement against the plain search, the fallback, invalid jobs.

The refinement evaluates each chosen cell's fine points with the exact
search's own per-point code, so its results are compared with the plain
search exactly: refining every cell of a grid is the full search, and on
the 0.025 m grid of the 12 x 9 m field it equals pps_propose bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1909_07717_gb300 import pps, synth

pytestmark = pytest.mark.gpu
PARAMS = dict(synth.DEFAULT_PARAMS)
SPEEDS = [2.0, 3.5, 5.0, 6.5]
BEST_FIELDS = ("idx", "ix", "iy", "speed_idx", "score", "margin", "status")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    return t


def _same_best(a, b):
    return all(a[f].tobytes() == b[f].tobytes() for f in BEST_FIELDS)


def _propose_jobs(torch, batch, spacing, weights, topk, flags=0, max_opp=16,
                  jobs=None):
    S = batch["ball"].shape[0]
    s = pps.Searcher(max_states=S, max_opp=max_opp)
    net = pps.Net(max_batch=S, weights=weights)
    try:
        dev = s.states_to_device(batch)
        if jobs is None:
            jobs = pps.field_jobs(batch, spacing, SPEEDS)
        dj = torch.from_numpy(pps.jobs_to_bytes(jobs)).cuda()
        best = torch.empty(S * 32, dtype=torch.uint8, device="cuda")
        cells = torch.empty((S, topk), dtype=torch.int32, device="cuda")
        pps.pps_propose_jobs(s.ctx, net.net, dev.data_ptr(), dj.data_ptr(), S,
                             spacing, len(SPEEDS), pps.params_from_dict(PARAMS),
                             topk, flags, best.data_ptr(), cells.data_ptr())
        torch.cuda.synchronize()
        pps.pps_net_sync(net.net)
        return pps.unpack_best(best.cpu().numpy()), cells.cpu().numpy()
    finally:
        net.close()
        s.close()


def _exact_per_field(torch, batch, spacing, max_opp=16):
    """The plain full-grid search of every state on its own field's grid
    (one pps_search per field size)."""
    S = batch["ball"].shape[0]
    out = np.zeros(S, pps.BEST_DTYPE)
    for L, W in {(float(a), float(b)) for a, b in
                 zip(batch["field_len"], batch["field_wid"])}:
        idx = np.flatnonzero((batch["field_len"] == L)
                             & (batch["field_wid"] == W))
        sub = synth.take(batch, idx)
        s = pps.Searcher(max_states=len(idx), max_opp=max_opp)
        try:
            grid = pps.pps_grid_from_field(L, W, spacing)
            o = s.search(s.states_to_device(sub), len(idx), grid, SPEEDS,
                         PARAMS, mask=False)
            torch.cuda.synchronize()
            out[idx] = pps.unpack_best(o["best"].cpu().numpy())
        finally:
            s.close()
    return out


def _lattice(grid):
    """(m, ox, oy) of a grid on the map's lattice: pixel (cx, cy) holds fine
    columns m cx + ox .. + m - 1 and rows m cy + oy .. + m - 1."""
    m = int(round(0.2 / float(np.float32(grid.spacing))))
    ox = int(round((-6.0 - grid.x0) / grid.spacing)) - m // 2
    oy = int(round((-4.5 - grid.y0) / grid.spacing)) - m // 2
    return m, ox, oy


def test_lattice_covers_every_point_once():
    """Each point of the served grids falls in exactly one map cell (the
    arithmetic of the kernels' lattice, restated)."""
    for L, W, g in ((12.0, 9.0, 0.025), (12.0, 9.0, 0.05), (9.0, 6.0, 0.05),
                    (12.0, 9.0, 0.1), (9.0, 6.0, 0.2)):
        grid = pps.pps_grid_from_field(L, W, g)
        m, ox, oy = _lattice(grid)
        count = np.zeros((grid.ny, grid.nx), np.int32)
        for cy in range(46):
            for cx in range(61):
                x0, y0 = m * cx + ox, m * cy + oy
                xs = slice(max(x0, 0), max(min(x0 + m, grid.nx), 0))
                ys = slice(max(y0, 0), max(min(y0 + m, grid.ny), 0))
                count[ys, xs] += 1
        assert np.all(count == 1), (L, W, g)


def test_equals_pps_propose_on_the_fine_12x9_grid(torch):
    """All jobs the 0.025 m grid of the 12 x 9 m field: the same cells, the
    same items in the same order, so without pruning the records equal
    pps_propose's byte for byte, and with it the best passes do."""
    batch = synth.ssl_states(701, 24, K=32)
    w = pps.load_net_weights()
    S = 24
    s = pps.Searcher(max_states=S, max_opp=8)
    net = pps.Net(max_batch=S, weights=w)
    try:
        dev = s.states_to_device(batch)
        ref = {}
        for flags in (pps.PPS_PROPOSE_NO_PRUNE, 0):
            best = torch.empty(S * 32, dtype=torch.uint8, device="cuda")
            pps.pps_propose(s.ctx, net.net, dev.data_ptr(), S,
                            pps.fine_grid_12x9(), SPEEDS,
                            pps.params_from_dict(PARAMS), 256, flags,
                            best.data_ptr(), None)
            torch.cuda.synchronize()
            ref[flags] = pps.unpack_best(best.cpu().numpy())
    finally:
        net.close()
        s.close()
    for flags in (pps.PPS_PROPOSE_NO_PRUNE, 0):
        got, _ = _propose_jobs(torch, batch, 0.025, w, 256, flags, max_opp=8)
        if flags:
            assert got.tobytes() == ref[flags].tobytes()
        else:
            assert _same_best(got, ref[flags])


def test_all_cells_of_mixed_fields_equal_the_full_search(torch):
    """12 x 9 and 9 x 6 m fields at 0.05 m, 6-11 opponents: refining every
    cell is the full search of each state's own grid."""
    batch = synth.serving_states(702, 12)
    best, _ = _propose_jobs(torch, batch, 0.05, pps.init_weights(3), 2806,
                            pps.PPS_PROPOSE_NO_PRUNE)
    ref = _exact_per_field(torch, batch, 0.05)
    assert _same_best(best, ref)
    assert np.array_equal(best["n_feasible"], ref["n_feasible"])
    pruned, _ = _propose_jobs(torch, batch, 0.05, pps.init_weights(3), 2806)
    assert _same_best(pruned, ref)


@pytest.mark.parametrize("max_opp", [16, 12])
def test_small_batches_split_points_across_lanes(torch, max_opp):
    """A batch too small to fill the GPU shares each point among several
    lanes (they split its samples and take the minimum across them; with at
    least as many lanes a point as opponent slots, the shot angle is formed
    across them too): one and two states refined alone give the bytes they
    get inside a 64-state batch, where every lane holds a point of its own.
    16 and 12 opponent slots (the states have 6 to 11 opponents)."""
    batch = synth.serving_states(707, 64)
    w = pps.load_net_weights(pps.SERVING_WEIGHTS)
    for flags in (pps.PPS_PROPOSE_NO_PRUNE, 0):
        big, big_cells = _propose_jobs(torch, batch, 0.05, w, 256, flags,
                                       max_opp=max_opp)
        for idx in ([5], [0, 1]):
            got, cells = _propose_jobs(torch, synth.take(batch, idx), 0.05, w,
                                       256, flags, max_opp=max_opp)
            assert np.array_equal(cells, big_cells[idx])
            if flags:
                assert got.tobytes() == big[idx].tobytes()
            else:
                assert _same_best(got, big[idx])


def test_off_grid_cells_rank_last(torch):
    """On a 9 x 6 m field only 46 x 31 of the map's cells hold points: the
    top cells are all among them, in the network's order."""
    batch = synth.serving_states(703, 6)
    k = 46 * 31
    _, cells = _propose_jobs(torch, batch, 0.05, pps.init_weights(4), k)
    for s in range(6):
        grid = pps.pps_grid_from_field(float(batch["field_len"][s]),
                                       float(batch["field_wid"][s]), 0.05)
        m, ox, oy = _lattice(grid)
        cy, cx = np.divmod(cells[s], 61)
        on = ((m * cx + ox + m > 0) & (m * cx + ox < grid.nx)
              & (m * cy + oy + m > 0) & (m * cy + oy < grid.ny))
        assert on.all(), s
        assert len(set(cells[s].tolist())) == k


def test_fallback_on_mixed_fields(torch):
    """A network that predicts 0 everywhere ranks the first cells of each
    grid (a corner) first; two cells per state miss many states' passes,
    and the fallback searches those states on their own full grids."""
    from tests.test_gpu_net import _cancel_weights
    batch = synth.serving_states(704, 20)
    no_fb, cells = _propose_jobs(torch, batch, 0.05, _cancel_weights(), 2)
    fb, _ = _propose_jobs(torch, batch, 0.05, _cancel_weights(), 2,
                          pps.PPS_PROPOSE_FALLBACK)
    ref = _exact_per_field(torch, batch, 0.05)
    missed = no_fb["idx"] == -1
    assert missed.any() and (~missed).any()
    assert fb[missed].tobytes() == ref[missed].tobytes()
    assert _same_best(fb[~missed], no_fb[~missed])


def test_jobs_that_do_not_fit_are_invalid(torch):
    """A job at another spacing, off the lattice, or with more speeds than
    max_speeds is flagged; the other states are unaffected."""
    batch = synth.serving_states(705, 4)
    jobs = pps.field_jobs(batch, 0.05, SPEEDS)
    jobs[1].grid = pps.pps_grid_from_field(12.0, 9.0, 0.1)     # spacing
    jobs[2].grid.x0 += 0.01                                    # off lattice
    jobs[3].n_speeds = 8                                       # > max_speeds
    for v in range(8):
        jobs[3].speeds[v] = 3.0
    best, _ = _propose_jobs(torch, batch, 0.05, pps.init_weights(5), 64,
                            pps.PPS_PROPOSE_FALLBACK, jobs=jobs)
    assert best["status"][0] == 0
    for i in (1, 2, 3):
        assert best["status"][i] & pps.PPS_STATE_INVALID and best["idx"][i] == -2


def test_labels_on_the_serving_grids(torch):
    """pps_net_labels_grid: per map pixel the best of its cell's points on
    the 0.05 m grids of both fields, floor where a cell holds no point."""
    rng = np.random.default_rng(706)
    for L, W in ((12.0, 9.0), (9.0, 6.0)):
        grid = pps.pps_grid_from_field(L, W, 0.05)
        pb = rng.normal(size=(2, grid.ny, grid.nx)).astype(np.float32)
        pb[pb < -1] = -np.inf
        net = pps.Net(max_batch=2)
        try:
            d = torch.from_numpy(pb).cuda()
            lab = torch.empty((2, 46, 61), dtype=torch.float32, device="cuda")
            pps.pps_net_labels_grid(net.net, d.data_ptr(), 2, grid, -1.2,
                                    lab.data_ptr())
            got = lab.cpu().numpy()
        finally:
            net.close()
        m, ox, oy = _lattice(grid)
        ref = np.full((2, 46, 61), -1.2, np.float32)
        for cy in range(46):
            for cx in range(61):
                ys = slice(max(m * cy + oy, 0), max(m * cy + oy + m, 0))
                xs = slice(max(m * cx + ox, 0), max(m * cx + ox + m, 0))
                blk = pb[:, ys, xs]
                if blk.size:
                    ref[:, cy, cx] = np.maximum(blk.max(axis=(1, 2)), -1.2)
        assert np.array_equal(got, ref), (L, W)
