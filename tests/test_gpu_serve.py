"""The serving loop (continuous batching) on the GPU.

Each test drives a pps_server through the C ABI: single frames alone and in
a mix of other matches' frames must get the same result; a replayed set of
simulated matches at 60 Hz must equal a batched-plan search of the same
frames (and the oracle on sampled frames); and the device-memory admission
budget must bound how many requests share a launch.
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
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    return t


def _server(streams=4, max_batch=256, pool=64 << 20, max_queue=16384,
            wait_us=50):
    d = pps.pps_server_desc(0, streams, max_batch, max_queue, pool, 16,
                            wait_us, pps.params_from_dict(PARAMS))
    return pps.pps_server_create(d)


def _reference(torch, frames, jobs):
    """The same frames through a batched plan (no graph, no tuning)."""
    S = frames["ball"].shape[0]
    s = pps.Searcher(max_states=S, max_opp=16)
    try:
        plan = pps.Plan(s, jobs, S, PARAMS, autotune=False, graph=False)
        plan.run(s.states_to_device(frames))
        torch.cuda.synchronize()
        best = pps.unpack_best(plan.best.cpu().numpy())
        mask = plan.mask.cpu().numpy().view(np.uint32)
        off = plan.offsets.copy()
        plan.close()
    finally:
        s.close()
    return best, mask, off


def _words(job):
    P = job.grid.nx * job.grid.ny
    return job.n_speeds * ((P + 31) // 32)


def test_alone_equals_in_the_mix(torch):
    frames = synth.serving_matches(401, 16, 8)
    rec = pps.pack_states(frames)
    jobs = pps.jobs_from_batch(frames)
    S = rec.shape[0]
    srv = _server()
    try:
        m0 = np.zeros(_words(jobs[5]), np.uint32)
        t = pps.pps_server_submit(srv, rec[5:6].ctypes.data,
                                  pps.ctypes.addressof(jobs[5]))
        alone = pps.pps_server_wait(srv, t, -1, m0)
        assert alone.batch_size == 1
        tickets = [pps.pps_server_submit(srv, rec[i:i + 1].ctypes.data,
                                         pps.ctypes.addressof(jobs[i]))
                   for i in range(S)]
        mixed = [pps.pps_server_wait(srv, t, -1,
                                     np.zeros(_words(jobs[i]), np.uint32))
                 for i, t in enumerate(tickets)]
        m5 = np.zeros(_words(jobs[5]), np.uint32)
        t = pps.pps_server_submit(srv, rec[5:6].ctypes.data,
                                  pps.ctypes.addressof(jobs[5]))
        again = pps.pps_server_wait(srv, t, -1, m5)
    finally:
        pps.pps_server_destroy(srv)
    assert max(r.batch_size for r in mixed) > 1, "no batching happened"
    assert bytes(alone.best) == bytes(mixed[5].best) == bytes(again.best)
    assert np.array_equal(m0, m5)
    ref, rmask, off = _reference(torch, frames, jobs)
    got = np.frombuffer(b"".join(bytes(r.best) for r in mixed),
                        pps.BEST_DTYPE)
    assert got.tobytes() == ref.tobytes()
    assert np.array_equal(m0, rmask[off[5]:off[6]])


def test_replay_matches_plan_and_oracle(torch):
    M, F = 32, 30
    frames = synth.serving_matches(402, M, F)
    rec = pps.pack_states(frames)
    jobs_m = pps.match_jobs(frames)
    srv = _server()
    try:
        res = np.zeros(M * F, pps.RESULT_DTYPE)
        st = pps.pps_server_replay(srv, rec, jobs_m, M, F, 60.0, res)
    finally:
        pps.pps_server_destroy(srv)
    assert st.completed == M * F
    assert np.all(res["status"] == 0)
    assert st.p99_us > 0 and st.p50_us <= st.p99_us <= st.max_us
    jobs = pps.jobs_from_batch(frames)
    ref, _, _ = _reference(torch, frames, jobs)
    assert res["best"].tobytes() == ref.tobytes()
    for i in (0, 7 * F + 3, M * F - 1):
        job = jobs[i]
        gs = (float(np.float32(job.grid.spacing)), job.grid.nx, job.grid.ny,
              float(np.float32(job.grid.x0)), float(np.float32(job.grid.y0)))
        speeds = [float(job.speeds[v]) for v in range(job.n_speeds)]
        sub = synth.take({k: v for k, v in frames.items()
                          if isinstance(v, np.ndarray)}, [i])
        orc = oracle.search(sub, gs, speeds, PARAMS, dense=True)
        parity.check_best({"best": res["best"][[i]]}, orc, 0, gs[1],
                          gs[1] * gs[2])


def test_admission_by_device_memory(torch):
    frames = synth.serving_matches(403, 20, 2)
    rec = pps.pack_states(frames)
    jobs = pps.jobs_from_batch(frames)
    words = [_words(jobs[i]) for i in range(rec.shape[0])]
    big = max(words)
    pick = [i for i in range(rec.shape[0]) if words[i] == big]
    assert len(pick) >= 8
    # each stream's share of the pool holds one largest request, not two
    srv = _server(streams=2, pool=2 * 4 * (big + big // 2))
    try:
        tickets = [pps.pps_server_submit(srv, rec[i:i + 1].ctypes.data,
                                         pps.ctypes.addressof(jobs[i]))
                   for i in pick]
        out = [pps.pps_server_wait(srv, t, -1) for t in tickets]
    finally:
        pps.pps_server_destroy(srv)
    assert all(r.status == 0 for r in out)
    assert all(r.batch_size == 1 for r in out)
    ref, _, _ = _reference(torch, frames, jobs)
    got = np.frombuffer(b"".join(bytes(r.best) for r in out), pps.BEST_DTYPE)
    assert got.tobytes() == ref[pick].tobytes()
    # a request whose mask can never fit is refused at submission
    tiny = _server(streams=1, pool=4 * 16)
    try:
        with pytest.raises(pps.PpsError) as e:
            pps.pps_server_submit(tiny, rec[0:1].ctypes.data,
                                  pps.ctypes.addressof(jobs[0]))
        assert e.value.status == pps.PPS_ENOMEM
    finally:
        pps.pps_server_destroy(tiny)


def test_bad_requests_are_refused(torch):
    frames = synth.serving_matches(404, 2, 1)
    rec = pps.pack_states(frames)
    jobs = pps.jobs_from_batch(frames)
    srv = _server()
    try:
        bad = rec.copy()
        bad["K"][0] = 0
        with pytest.raises(pps.PpsError) as e:
            pps.pps_server_submit(srv, bad[0:1].ctypes.data,
                                  pps.ctypes.addressof(jobs[0]))
        assert e.value.status == pps.PPS_EINVAL
        jobs[1].n_speeds = 0
        with pytest.raises(pps.PpsError):
            pps.pps_server_submit(srv, rec[1:2].ctypes.data,
                                  pps.ctypes.addressof(jobs[1]))
        with pytest.raises(pps.PpsError) as e:
            pps.pps_server_wait(srv, 123456, 1000)
        assert e.value.status == pps.PPS_ETIMEOUT
    finally:
        pps.pps_server_destroy(srv)


# ------------------------------------------------------------ proposal mode
BEST_FIELDS = ("idx", "ix", "iy", "speed_idx", "score", "margin", "status")


def _proposal_server(weights, streams=4, max_batch=256, topk=256,
                     wait_us=50):
    w = np.ascontiguousarray(weights, np.float32)
    d = pps.pps_server_desc(0, streams, max_batch, 16384, 0, 16, wait_us,
                            pps.params_from_dict(PARAMS),
                            pps.PPS_SERVE_PROPOSAL, topk, w.ctypes.data)
    return pps.pps_server_create(d)   # the weights are copied


def _best_fields(best):
    return [best[f].tobytes() for f in BEST_FIELDS]


def _propose_direct(torch, frames, jobs, weights, topk=256):
    """The same frames through pps_propose_jobs (with the fallback)."""
    from paper_1909_07717_gb300.proposal import JobsProposal
    S = frames["ball"].shape[0]
    pr = JobsProposal(S, weights)
    try:
        st = pr.searcher.states_to_device(
            {k: v for k, v in frames.items() if isinstance(v, np.ndarray)})
        b, _ = pr.run(st, pr.jobs_to_device(jobs), S, topk=topk)
        torch.cuda.synchronize()
        return pps.unpack_best(b.cpu().numpy())
    finally:
        pr.close()


def test_proposal_alone_equals_in_the_mix(torch):
    """Proposal mode: a frame alone, in a mix of 128 frames of 16 matches
    and alone again gets the same best pass, and every frame the one
    pps_propose_jobs gives it (fields, grids and speeds of its own)."""
    frames = synth.serving_matches(405, 16, 8)
    rec = pps.pack_states(frames)
    jobs = pps.jobs_from_batch(frames)
    S = rec.shape[0]
    w = pps.load_net_weights(pps.SERVING_WEIGHTS)
    srv = _proposal_server(w)
    try:
        def one(i):
            t = pps.pps_server_submit(srv, rec[i:i + 1].ctypes.data,
                                      pps.ctypes.addressof(jobs[i]))
            return pps.pps_server_wait(srv, t, -1)
        alone = one(5)
        assert alone.batch_size == 1
        tickets = [pps.pps_server_submit(srv, rec[i:i + 1].ctypes.data,
                                         pps.ctypes.addressof(jobs[i]))
                   for i in range(S)]
        mixed = [pps.pps_server_wait(srv, t, -1) for t in tickets]
        again = one(5)
    finally:
        pps.pps_server_destroy(srv)
    assert max(r.batch_size for r in mixed) > 1, "no batching happened"
    got = np.frombuffer(b"".join(bytes(r.best) for r in mixed),
                        pps.BEST_DTYPE)
    a = np.frombuffer(bytes(alone.best), pps.BEST_DTYPE)
    b = np.frombuffer(bytes(again.best), pps.BEST_DTYPE)
    assert _best_fields(a) == _best_fields(got[5:6]) == _best_fields(b)
    assert np.all(got["status"] == 0)
    ref = _propose_direct(torch, frames, jobs, w)
    assert _best_fields(got) == _best_fields(ref)


def test_proposal_replay_agrees_with_the_exact_search(torch):
    """60 Hz replay of 32 matches in the proposal mode: every frame served,
    each result what pps_propose_jobs gives, never above the exact best,
    and within 2 % of it on at least 99 % of the frames."""
    from paper_1909_07717_gb300.proposal import agreement
    M, F = 32, 30
    frames = synth.serving_matches(406, M, F)
    rec = pps.pack_states(frames)
    jobs_m = pps.match_jobs(frames)
    w = pps.load_net_weights(pps.SERVING_WEIGHTS)
    srv = _proposal_server(w)
    try:
        res = np.zeros(M * F, pps.RESULT_DTYPE)
        st = pps.pps_server_replay(srv, rec, jobs_m, M, F, 60.0, res)
    finally:
        pps.pps_server_destroy(srv)
    assert st.completed == M * F and np.all(res["status"] == 0)
    jobs = pps.jobs_from_batch(frames)
    got = res["best"]
    assert _best_fields(got) == _best_fields(
        _propose_direct(torch, frames, jobs, w))
    ex, _, _ = _reference(torch, frames, jobs)
    found = got["idx"] >= 0
    assert np.all(got["score"][found] <= ex["score"][found])
    ok = agreement(got, ex)
    assert ok.mean() >= 0.99, ok.mean()


def test_proposal_mode_refuses_what_it_cannot_serve(torch):
    frames = synth.serving_matches(407, 2, 1)
    rec = pps.pack_states(frames)
    jobs = pps.jobs_from_batch(frames)
    d = pps.pps_server_desc(0, 1, 8, 64, 0, 16, 0,
                            pps.params_from_dict(PARAMS),
                            pps.PPS_SERVE_PROPOSAL, 256, None)
    with pytest.raises(pps.PpsError) as e:
        pps.pps_server_create(d)
    assert e.value.status == pps.PPS_EINVAL
    srv = _proposal_server(pps.init_weights(1), streams=1, max_batch=8)
    try:
        jobs[0].grid.x0 += 0.01          # off the map's cell lattice
        with pytest.raises(pps.PpsError) as e:
            pps.pps_server_submit(srv, rec[0:1].ctypes.data,
                                  pps.ctypes.addressof(jobs[0]))
        assert e.value.status == pps.PPS_EINVAL
        t = pps.pps_server_submit(srv, rec[1:2].ctypes.data,
                                  pps.ctypes.addressof(jobs[1]))
        assert pps.pps_server_wait(srv, t, -1).status == 0
    finally:
        pps.pps_server_destroy(srv)
