"""Batched plans (uneven batches) on the GPU against pps_search and the
FP64 oracle.

An uneven batch mixes 12 x 9 m fields with 11 opponents and 9 x 6 m fields
with 6, per-state grid spacings, 1-8 kick speeds, K from 32 to 128 and the
ball deceleration in [0.3, 0.7].  A plan groups the states by kernel
instance; these tests check that grouping, the per-state mask layout, the
autotuner and the CUDA-graph replay leave every state's result equal to the
definition.
"""
from __future__ import annotations

import ctypes

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
    s = pps.Searcher(max_states=8192, max_opp=16, max_K=256)
    yield s
    s.close()


def _plan_run(searcher, batch, jobs, autotune=True, graph=True, runs=1):
    S = batch["ball"].shape[0]
    plan = pps.Plan(searcher, jobs, S, PARAMS, autotune=autotune, graph=graph)
    st = searcher.states_to_device(batch)
    for _ in range(runs):
        plan.run(st)
    searcher.torch.cuda.synchronize()
    best = pps.unpack_best(plan.best.cpu().numpy())
    mask = plan.mask.cpu().numpy().view(np.uint32)
    groups = plan.groups()
    off = plan.offsets.copy()
    plan.close()
    return best, mask, off, groups


def _gspec(job):
    g = job.grid
    return (float(np.float32(g.spacing)), g.nx, g.ny, float(np.float32(g.x0)),
            float(np.float32(g.y0)))


def _check_state(best, mask, off, jobs, batch, s):
    job = jobs[s]
    V = job.n_speeds
    speeds = [float(job.speeds[v]) for v in range(V)]
    gs = _gspec(job)
    P = gs[1] * gs[2]
    sub = synth.take(batch, [s])
    orc = oracle.search(sub, gs, speeds, PARAMS, dense=True)
    bits = parity.words_to_bits(mask[off[s]:off[s + 1]], V, P)
    st = oracle.state_of(sub, 0)
    parity.check_mask_one(bits, orc["feasible"][0], orc["margin"][0], st, gs,
                          speeds, PARAMS)
    assert bits.sum() == best[s]["n_feasible"]
    parity.check_best({"best": best[[s]]}, orc, 0, gs[1], P)


def test_plan_equals_search_on_a_uniform_batch(searcher):
    batch = synth.ssl_states(301, 12, K=32)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.2)
    speeds = [2.0, 3.5, 5.0, 6.5]
    ref = parity.run_gpu(searcher, batch, grid, speeds, PARAMS, debug=False,
                         T=False)
    jobs = (pps.pps_job * 12)()
    for i in range(12):
        jobs[i].grid = grid
        jobs[i].n_speeds = 4
        for v in range(4):
            jobs[i].speeds[v] = speeds[v]
        jobs[i].max_opp = 8
    best, mask, off, groups = _plan_run(searcher, batch, jobs)
    assert best.tobytes() == ref["best"].tobytes()
    assert np.array_equal(mask[:off[-1]], ref["mask"])
    assert len(groups) == 1 and groups[0].opp_slots == 8


def test_uneven_plan_parity(searcher):
    """Small uneven batch, every state against the oracle."""
    batch = synth.uneven_batch(302, 24, spacings=(0.2, 0.3, 0.5),
                               k_range=(32, 128))
    jobs = pps.jobs_from_batch(batch)
    best, mask, off, groups = _plan_run(searcher, batch, jobs)
    assert {(g.opp_slots) for g in groups} == {6, 12}
    assert sum(g.n_states for g in groups) == 24
    assert np.all(best["status"] == 0)
    for s in range(24):
        _check_state(best, mask, off, jobs, batch, s)


def test_plan_without_graph_or_tuning_matches(searcher):
    batch = synth.uneven_batch(303, 16, spacings=(0.25, 0.5))
    jobs = pps.jobs_from_batch(batch)
    a = _plan_run(searcher, batch, jobs, autotune=True, graph=True, runs=3)
    b = _plan_run(searcher, batch, jobs, autotune=False, graph=False)
    assert a[0].tobytes() == b[0].tobytes()
    assert np.array_equal(a[1], b[1])


def test_graph_replay_follows_buffer_contents(searcher):
    """A captured graph re-reads the states buffer on every replay."""
    torch = searcher.torch
    b1 = synth.uneven_batch(304, 10, spacings=(0.25, 0.5))
    b2 = synth.uneven_batch(305, 10, spacings=(0.25, 0.5))
    for k in ("spacing", "n_speeds", "speeds", "n_opp", "field_len",
              "field_wid", "goal_width"):
        b2[k] = b1[k]   # same shapes, different positions
    jobs = pps.jobs_from_batch(b1)
    plan = pps.Plan(searcher, jobs, 10, PARAMS, autotune=False, graph=True)
    st = searcher.states_to_device(b1)
    plan.run(st)
    torch.cuda.synchronize()
    first = plan.best.cpu().numpy().copy()
    st.copy_(searcher.states_to_device(b2))
    plan.run(st)
    torch.cuda.synchronize()
    second = pps.unpack_best(plan.best.cpu().numpy())
    plan.close()
    ref = _plan_run(searcher, b2, jobs, autotune=False, graph=False)[0]
    assert second.tobytes() == ref.tobytes()
    assert first.tobytes() != second.tobytes()


def test_plan_rejects_bad_jobs(searcher):
    jobs = (pps.pps_job * 2)()
    for i in range(2):
        jobs[i].grid = pps.pps_grid_from_field(12.0, 9.0, 0.5)
        jobs[i].n_speeds = 1
        jobs[i].speeds[0] = 3.0
        jobs[i].max_opp = 8
    for field, value in [("n_speeds", 0), ("n_speeds", 9), ("max_opp", 17)]:
        bad = (pps.pps_job * 2)()
        ctypes.memmove(bad, bytes(jobs), len(bytes(jobs)))
        setattr(bad[1], field, value)
        with pytest.raises(pps.PpsError) as e:
            pps.pps_plan_create(searcher.ctx, bad, 2)
        assert e.value.status == pps.PPS_EINVAL
    bad = (pps.pps_job * 2)()
    ctypes.memmove(bad, bytes(jobs), len(bytes(jobs)))
    bad[0].speeds[0] = -1.0
    with pytest.raises(pps.PpsError):
        pps.pps_plan_create(searcher.ctx, bad, 2)


# -------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def full_uneven(searcher):
    batch = synth.uneven_batch(synth.UNEVEN_SEED, synth.UNEVEN_STATES)
    jobs = pps.jobs_from_batch(batch)
    best, mask, off, groups = _plan_run(searcher, batch, jobs, runs=2)
    return batch, jobs, best, mask, off, groups


def test_uneven_full_size_properties(full_uneven):
    batch, jobs, best, mask, off, groups = full_uneven
    S = synth.UNEVEN_STATES
    assert np.all(best["status"] == 0)
    assert all(g.cta_threads in (128, 256, 512, 768, 1024) for g in groups)
    # samples a register block: 2 only at the two smallest CTA sizes
    assert all(g.sample_unroll == 1 or (g.sample_unroll == 2 and
                                        g.cta_threads in (128, 256))
               for g in groups)
    has = best["idx"] >= 0
    assert np.all(has == (best["n_feasible"] > 0))
    for s in range(0, S, 97):      # popcounts and best bits, spread over all
        job = jobs[s]
        P = job.grid.nx * job.grid.ny
        bits = parity.words_to_bits(mask[off[s]:off[s + 1]], job.n_speeds, P)
        assert bits.sum() == best[s]["n_feasible"]
        if has[s]:
            assert bits.reshape(-1)[best[s]["idx"]]


def test_uneven_full_size_sampled_states(full_uneven):
    """States of the full batch whose oracle cost is a few seconds."""
    batch, jobs, best, mask, off, groups = full_uneven
    cost = np.array([jobs[s].grid.nx * jobs[s].grid.ny * jobs[s].n_speeds
                     * int(batch["K"][s]) * int(batch["n_opp"][s])
                     for s in range(synth.UNEVEN_STATES)])
    pick = [s for s in range(synth.UNEVEN_STATES) if cost[s] < 4e7][:: 97][:8]
    assert len(pick) >= 6
    for s in pick:
        _check_state(best, mask, off, jobs, batch, s)
