"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Sizes: the single-state workload whole (121 x 91 grid, 87 tiles of 128
points with a ragged last tile), a multi-state batch with the batched
workload's shape on a coarser grid, edge cases, and the full batched
workload (4096 x 241 x 181, 4 speeds, K = 64) in the benchmark's launch
configuration, checked on sampled states against the oracle and on every
state through properties that hold at any size.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1909_07717_gb300 import pps, synth
from tests import parity

pytestmark = pytest.mark.gpu

PARAMS = dict(synth.DEFAULT_PARAMS)


@pytest.fixture(scope="module")
def searcher():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    s = pps.Searcher(max_states=4096, max_opp=8, max_K=256)
    yield s
    s.close()


@pytest.fixture(scope="module")
def searcher16():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = pps.Searcher(max_states=64, max_opp=16, max_K=256)
    yield s
    s.close()


def _dense_case(searcher, batch, grid, speeds, params=PARAMS, states=None):
    gpu = parity.run_gpu(searcher, batch, grid, speeds, params)
    orc = oracle.search(batch, parity.grid_spec(grid), speeds, params,
                        dense=True, want_T=True)
    S = batch["ball"].shape[0]
    P = grid.nx * grid.ny
    stats = []
    for s in (range(S) if states is None else states):
        stats.append(parity.check_state_dense(gpu, orc, batch, s, grid,
                                              speeds, params))
        parity.check_best(gpu, orc, s, grid.nx, P)
        # the counts can differ only by candidates inside the mask's bands
        nf_o = int(orc["n_feasible"][s])
        nf_g = int(gpu["best"][s]["n_feasible"])
        assert abs(nf_g - nf_o) <= stats[-1]["mask_band_count"], (
            nf_g, nf_o, stats[-1]["mask_band_count"])
        mask, _ = parity.unpack_mask(gpu["mask"], S, len(speeds), P)
        assert mask[s].sum() == nf_g
    return gpu, orc, stats


def test_single_state_workload(searcher):
    """12x9 m, 0.1 m grid, one speed 4 m/s, K = 32, 8 opponents."""
    w = synth.SINGLE
    batch = w.states()
    grid = pps.pps_grid_from_field(12.0, 9.0, w.spacing)
    assert (grid.nx, grid.ny) == (121, 91)
    assert parity.grid_spec(grid)[1:3] == oracle.grid(12.0, 9.0,
                                                      np.float32(0.1))[:2]
    gpu, orc, stats = _dense_case(searcher, batch, grid, w.speeds)
    print(stats)


def test_batched_shape_small_grid(searcher):
    """Batched workload shape (4 speeds, K = 64, 8 v 8) on a 0.2 m grid."""
    w = synth.BATCHED
    batch = synth.ssl_states(101, 6, K=64)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.2)
    _, orc, stats = _dense_case(searcher, batch, grid, w.speeds)
    print(stats)


def test_marked_layout(searcher):
    """Opponents marking receivers: the mixed-feasibility regime."""
    batch = synth.ssl_states(102, 4, K=32, marked=True)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.25)
    _dense_case(searcher, batch, grid, [2.0, 3.5, 5.0, 6.5])


@pytest.mark.parametrize("speeds", [[3.0], [2.0, 6.0], [2.0, 3.0, 4.0],
                                    [1.5, 2.5, 3.5, 4.5, 5.5],
                                    [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 6.5, 7.0]])
def test_speed_counts(searcher, speeds):
    batch = synth.ssl_states(103, 2, K=16)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.4)
    _dense_case(searcher, batch, grid, speeds)


@pytest.mark.parametrize("K", [1, 2, 37, 128])
def test_sample_counts(searcher, K):
    batch = synth.ssl_states(104, 2, K=K)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.4)
    _dense_case(searcher, batch, grid, [2.5, 5.0])


def test_mixed_opponent_counts(searcher):
    batch = synth.ssl_states(105, 9, K=16)
    batch["n_opp"] = np.arange(9, dtype=np.int32)  # 0..8 opponents
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.3)
    gpu, orc, _ = _dense_case(searcher, batch, grid, [3.0, 5.0])
    # with no opponents every reachable pass is feasible, margins +inf
    assert np.all(np.isposinf(gpu["margin"][0][np.isfinite(
        orc["margin"][0]) | np.isposinf(orc["margin"][0])]))


def test_fast_opponents_clamp(searcher):
    """Opponents faster than vmax take the clamped path."""
    batch = synth.ssl_states(106, 3, K=16)
    batch["opp_vel"] *= 1.8
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.3)
    _dense_case(searcher, batch, grid, [3.0, 5.0])


def test_reach_radius_and_thresholds(searcher):
    batch = synth.ssl_states(107, 3, K=16)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.3)
    prm = dict(PARAMS, reach_radius=0.09, tau_safe=0.2, min_pass_dist=1.0,
               w_angle=0.7, w_dist=1.3, w_margin=2.0, margin_cap=0.6)
    _dense_case(searcher, batch, grid, [3.0, 5.0], params=prm)


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 5), (33, 4), (129, 1),
                                   (16, 16)])
def test_ragged_grids(searcher, nx, ny):
    batch = synth.ssl_states(108, 3, K=8)
    grid = pps.pps_grid(0.37, nx, ny, -5.1, -3.3)
    _dense_case(searcher, batch, grid, [2.0, 4.0, 6.0])


def test_coincident_points(searcher):
    """An opponent exactly on a grid point, and the ball on a grid point."""
    batch = synth.ssl_states(109, 2, K=8)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.5)
    batch["opp_pos"][0, 0] = [np.float32(-6.0 + 10 * np.float32(0.5)),
                              np.float32(-4.5 + 4 * np.float32(0.5))]
    batch["ball"][1] = [np.float32(-6.0 + 3 * np.float32(0.5)),
                        np.float32(-4.5 + 9 * np.float32(0.5))]
    _dense_case(searcher, batch, grid, [2.0, 4.0])


def test_sixteen_opponents(searcher16):
    """11 v 11 and 16-opponent states on the 16-slot kernel."""
    b1 = synth.ssl_states(110, 2, n_opp=11, K=32)
    b2 = synth.ssl_states(111, 2, n_opp=16, K=32)
    batch = synth.concat([b1, b2])
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.3)
    _dense_case(searcher16, batch, grid, [3.0, 5.0, 6.5])


def test_host_pointer_path_matches_device(searcher):
    batch = synth.ssl_states(112, 5, K=32)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.25)
    sp = [2.0, 3.5, 5.0, 6.5]
    d = parity.run_gpu(searcher, batch, grid, sp, PARAMS, debug=False,
                       T=False)
    h = parity.run_gpu(searcher, batch, grid, sp, PARAMS, host=True)
    assert d["best"].tobytes() == h["best"].tobytes()
    assert np.array_equal(d["mask"], h["mask"])


def test_deterministic(searcher):
    batch = synth.ssl_states(113, 7, K=32)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.2)
    sp = [2.0, 3.5, 5.0, 6.5]
    a = parity.run_gpu(searcher, batch, grid, sp, PARAMS)
    b = parity.run_gpu(searcher, batch, grid, sp, PARAMS)
    for k in a:
        assert np.asarray(a[k]).tobytes() == np.asarray(b[k]).tobytes(), k


def test_device_state_validation(searcher):
    """Invalid device-memory states are flagged; the others still run."""
    import torch
    batch = synth.ssl_states(114, 4, K=8)
    batch["n_opp"][1] = 12            # above the context's max_opp = 8
    batch["ball_decel"][2] = -1.0     # non-positive deceleration
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.5)
    gpu = parity.run_gpu(searcher, batch, grid, [3.0], PARAMS, debug=False,
                         T=False)
    st = gpu["best"]["status"]
    assert st[1] == pps.PPS_STATE_INVALID and st[2] == pps.PPS_STATE_INVALID
    assert gpu["best"]["idx"][1] == -2 and gpu["best"]["idx"][2] == -2
    assert st[0] == 0 and st[3] == 0
    ok = synth.take(batch, [0, 3])
    ref = parity.run_gpu(searcher, ok, grid, [3.0], PARAMS, debug=False,
                         T=False)
    assert ref["best"][0].tobytes() == gpu["best"][0].tobytes()
    assert ref["best"][1].tobytes() == gpu["best"][3].tobytes()
    # the same states from host memory are rejected before any work
    with pytest.raises(pps.PpsError) as e:
        parity.run_gpu(searcher, batch, grid, [3.0], PARAMS, host=True)
    assert e.value.status == pps.PPS_EINVAL
    torch.cuda.synchronize()


def _call(searcher, rec, n, grid, speeds, params):
    sp = np.asarray(speeds, np.float32)
    best = np.zeros(max(n, 1), pps.BEST_DTYPE)
    return pps.pps_search(searcher.ctx,
                          None if rec is None else rec.ctypes.data, n, grid,
                          sp.ctypes.data if len(sp) else None, len(sp),
                          pps.params_from_dict(params), best.ctypes.data,
                          None)


def test_argument_errors(searcher):
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.5)
    rec = pps.pack_states(synth.ssl_states(115, 2, K=8))
    cases = [
        (rec, 2, pps.pps_grid(-1.0, 3, 3, 0.0, 0.0), [3.0], PARAMS),
        (rec, 2, pps.pps_grid(0.1, 0, 3, 0.0, 0.0), [3.0], PARAMS),
        (rec, 2, grid, [], PARAMS),
        (rec, 2, grid, [0.0], PARAMS),
        (rec, 2, grid, [float("nan")], PARAMS),
        (rec, 2, grid, [1.0] * 9, PARAMS),
        (rec, 2, grid, [3.0], dict(PARAMS, reach_radius=-1.0)),
        (rec, 2, grid, [3.0], dict(PARAMS, w_angle=float("inf"))),
        (rec, 5000, grid, [3.0], PARAMS),
        (None, 2, grid, [3.0], PARAMS),
    ]
    for rec_, n, g, sp, prm in cases:
        with pytest.raises(pps.PpsError) as e:
            _call(searcher, rec_, n, g, sp, prm)
        assert e.value.status == pps.PPS_EINVAL
        assert pps.pps_last_error(searcher.ctx)
    bad = rec.copy()
    bad["K"][1] = 0
    with pytest.raises(pps.PpsError):
        _call(searcher, bad, 2, grid, [3.0], PARAMS)
    bad = rec.copy()
    bad["opp_pos"][0, 0, 0] = np.nan
    with pytest.raises(pps.PpsError):
        _call(searcher, bad, 2, grid, [3.0], PARAMS)
    # an empty batch is a no-op
    _call(searcher, None, 0, grid, [3.0], PARAMS)
    searcher.sync()


def test_memory_budget():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(pps.PpsError) as e:
        pps.pps_create(pps.pps_ctx_desc(max_states=1 << 20,
                                        mem_budget_bytes=1024))
    assert e.value.status == pps.PPS_ENOMEM
    s = pps.Searcher(max_states=8, mem_budget_bytes=100_000)
    try:
        batch = synth.ssl_states(116, 8, K=8)
        grid = pps.pps_grid_from_field(12.0, 9.0, 0.05)  # 89 KB of mask/state
        rec = pps.pack_states(batch)
        best = np.zeros(8, pps.BEST_DTYPE)
        mask = np.zeros(8 * pps.pps_mask_words(grid, 4), np.uint32)
        with pytest.raises(pps.PpsError) as e:
            s.search_host(rec, grid, [2.0, 3.5, 5.0, 6.5], PARAMS, best, mask)
        assert e.value.status == pps.PPS_ENOMEM
    finally:
        s.close()


# ------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def full_batched(searcher):
    """The batched workload at full size, as the benchmark launches it."""
    import torch
    w = synth.BATCHED
    batch = w.states()
    grid = pps.pps_grid_from_field(12.0, 9.0, w.spacing)
    st = searcher.states_to_device(batch)
    out = searcher.search(st, w.n_states, grid, w.speeds, w.params)
    torch.cuda.synchronize()
    best = pps.unpack_best(out["best"].cpu().numpy())
    mask = out["mask"].cpu().numpy().view(np.uint32)
    return w, batch, grid, best, mask


def test_full_size_properties(full_batched):
    """Properties at any size, on all 4096 states."""
    w, batch, grid, best, mask = full_batched
    S, V, P = w.n_states, len(w.speeds), grid.nx * grid.ny
    assert (grid.nx, grid.ny) == (241, 181)
    bits, pad = parity.unpack_mask(mask, S, V, P)
    assert not pad.any()
    assert np.all(best["status"] == 0)
    assert np.array_equal(bits.sum(axis=(1, 2)), best["n_feasible"])
    has = best["idx"] >= 0
    assert np.all(has == (best["n_feasible"] > 0))
    flat = bits.reshape(S, -1)
    assert np.all(flat[np.flatnonzero(has), best["idx"][has]])
    assert np.all(np.isfinite(best["score"][has]))
    assert np.all(best["margin"][has] > PARAMS["tau_safe"])


def test_full_size_sampled_states(full_batched):
    """Sampled states of the full batch against the oracle, densely."""
    w, batch, grid, best, mask = full_batched
    S, V, P = w.n_states, len(w.speeds), grid.nx * grid.ny
    pick = [0, 1, 977, 2048, 3001, 4095]
    sub = synth.take(batch, pick)
    orc = oracle.search(sub, parity.grid_spec(grid), w.speeds, w.params,
                        dense=True)
    bits, _ = parity.unpack_mask(mask, S, V, P)
    for i, s in enumerate(pick):
        gpu_i = {"best": best[[s]],
                 "mask": mask.reshape(S, -1)[s]}
        orc_i = {k: v[[i]] for k, v in orc.items()}
        st = oracle.state_of(sub, i)
        # mask outside the bands
        m_o = orc_i["margin"][0]
        _, cx, cy = parity.sample_points(st, grid, 1)
        D = np.hypot(cx - st.sc[0], cy - st.sc[1])
        sp = np.asarray(w.speeds, np.float64)
        gap = np.abs(sp[:, None] ** 2 - 2 * st.sc[2] * D[None, :]) / \
            sp[:, None] ** 2
        band = (np.abs(m_o) <= parity.TOL_MASK) | (gap <= parity.TOL_REACH)
        diff = (bits[s] != orc_i["feasible"][0].astype(bool)) & ~band
        assert not diff.any(), f"state {s}: {diff.sum()} mask bits differ"
        parity.check_best(gpu_i, orc_i, 0, grid.nx, P)
