"""Every entry point writes inside its output buffers and nowhere else.

compute-sanitizer is not available on the GPU pool, so out-of-bounds writes
are caught the plain way: each output buffer is allocated with 4 KiB of
canary bytes before and after it, every entry point runs on ragged shapes
(state counts and grids that are not multiples of 32, partial mask words,
empty teams), and the canaries must come back untouched.  Outputs whose
size the caller states exactly (mask words, dense planes) are also checked
to be fully written where the contract says so.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1909_07717_gb300 import pps, synth

pytestmark = pytest.mark.gpu
PAD = 4096
CANARY = 0xA5


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07717_gb300 import build
    build.build()
    return t


class Guarded:
    """nbytes of device memory between two canary regions."""

    def __init__(self, torch, nbytes, fill=CANARY):
        self.torch = torch
        self.n = int(nbytes)
        self.buf = torch.full((self.n + 2 * PAD,), CANARY, dtype=torch.uint8,
                              device="cuda")
        self.buf[PAD:PAD + self.n] = fill      # the body may start otherwise

    @property
    def ptr(self):
        return self.buf.data_ptr() + PAD

    def body(self):
        return self.buf[PAD:PAD + self.n].cpu().numpy()

    def intact(self):
        self.torch.cuda.synchronize()
        b = self.buf.cpu().numpy()
        return bool(np.all(b[:PAD] == CANARY) and np.all(b[PAD + self.n:] == CANARY))


def _dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8)
                            .reshape(-1).copy()).cuda()


def test_search_outputs_stay_in_bounds(torch):
    n, V, K = 37, 3, 17
    batch = synth.ssl_states(61, n, n_opp=7, K=K)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.3)       # 41 x 31: ragged
    P = grid.nx * grid.ny
    words = (P + 31) // 32
    s = pps.Searcher(max_states=64, max_opp=8)
    try:
        st = s.states_to_device(batch)
        best = Guarded(torch, n * 32)
        mask = Guarded(torch, n * V * words * 4)
        dm = Guarded(torch, n * V * P * 4)
        ds = Guarded(torch, n * V * P * 4)
        dT = Guarded(torch, n * P * K * 4)
        pb = Guarded(torch, n * P * 4)
        dbg = pps.pps_debug_out(dm.ptr, ds.ptr, dT.ptr, K, pb.ptr)
        sp = np.array([2.0, 4.0, 6.0], np.float32)
        pps.pps_search(s.ctx, st.data_ptr(), n, grid, sp.ctypes.data, V,
                       pps.params_from_dict(synth.DEFAULT_PARAMS), best.ptr,
                       mask.ptr, dbg, pps.PPS_DEVICE_PTRS)
        for g in (best, mask, dm, ds, dT, pb):
            assert g.intact()
        # every mask word and every debug value was written
        m = Guarded(torch, n * V * words * 4, fill=0x5A)
        pps.pps_search(s.ctx, st.data_ptr(), n, grid, sp.ctypes.data, V,
                       None, best.ptr, m.ptr, None, pps.PPS_DEVICE_PTRS)
        torch.cuda.synchronize()
        words_arr = m.body().view(np.uint32).reshape(n, V, words)
        tail = P - 32 * (words - 1)
        assert np.all(words_arr[:, :, -1] >> tail == 0)   # no bits past P
        assert m.intact()
    finally:
        s.close()


def test_noalloc_outputs_stay_in_bounds(torch):
    n = 19
    batch = synth.ssl_states(62, n, n_opp=5, K=9)
    grid = pps.pps_grid_from_field(9.0, 6.0, 0.25)
    words = (grid.nx * grid.ny + 31) // 32
    st = _dev(torch, pps.pack_states(batch))
    best = Guarded(torch, n * 32)
    mask = Guarded(torch, n * 2 * words * 4)
    sp = np.array([3.0, 5.0], np.float32)
    pps.pps_search_noalloc(0, None, 8, st.data_ptr(), n, grid, sp.ctypes.data,
                           2, None, best.ptr, mask.ptr)
    assert best.intact() and mask.intact()


def test_plan_outputs_stay_in_bounds(torch):
    batch = synth.uneven_batch(63, 45)
    jobs = pps.jobs_from_batch(batch)
    s = pps.Searcher(max_states=64, max_opp=16)
    try:
        plan = pps.pps_plan_create(s.ctx, jobs, 45, None,
                                   pps.PPS_PLAN_AUTOTUNE | pps.PPS_PLAN_GRAPH)
        try:
            off = pps.pps_plan_mask_offsets(plan, 45, s.ctx)
            st = _dev(torch, pps.pack_states(batch))
            best = Guarded(torch, 45 * 32)
            mask = Guarded(torch, int(off[-1]) * 4)
            for _ in range(2):       # tuned and captured, then replayed
                pps.pps_plan_run(plan, st.data_ptr(), best.ptr, mask.ptr,
                                 s.ctx)
                assert best.intact() and mask.intact()
        finally:
            pps.pps_plan_destroy(plan)
    finally:
        s.close()


def test_decision_outputs_stay_in_bounds(torch):
    n = 5
    batch = synth.dpps_states(64, n, n_team=3, n_opp=9, K=11)
    batch["n_team"] = batch["n_team"].copy()
    batch["n_team"][1] = 0
    prm = dict(synth.DPPS_PARAMS, n_dir=13, n_pow=21)      # partial words
    p = pps.dparams_from_dict(prm)
    C = 13 * 21
    s = pps.Searcher(max_states=8, max_opp=16)
    try:
        st = _dev(torch, pps.pack_dstates(batch))
        best = Guarded(torch, n * 48)
        mask = Guarded(torch, n * pps.pps_dpps_mask_words(p) * 4)
        dbg = Guarded(torch, n * C * 12)
        pps.pps_dpps_search(s.ctx, st.data_ptr(), n, p, best.ptr, mask.ptr,
                            dbg.ptr)
        assert best.intact() and mask.intact() and dbg.intact()
        # passing powers and shots
        q = np.zeros(29, pps.PASS_QUERY_DTYPE)
        q["state"] = np.arange(29) % n
        q["receiver"] = np.arange(29) % 3
        q["target"] = np.stack([np.linspace(-5, 5, 29), np.zeros(29)], 1)
        out = Guarded(torch, 29 * pps.PASS_POWER_DTYPE.itemsize)
        pps.pps_pass_powers(s.ctx, st.data_ptr(), n, _dev(torch, q).data_ptr(),
                            29, 0.3, p, out.ptr)
        assert out.intact()
        sq = np.zeros(31, pps.SHOT_QUERY_DTYPE)
        sq["state"] = np.arange(31) % n
        sq["from"] = np.stack([np.linspace(-2, 5.9, 31), np.zeros(31)], 1)
        sout = Guarded(torch, 31 * pps.SHOT_DTYPE.itemsize)
        pps.pps_shoot(s.ctx, st.data_ptr(), n, _dev(torch, sq).data_ptr(), 31,
                      6.5, 0.1, p, sout.ptr)
        assert sout.intact()
        # running points avoiding the best passes, with dense scores
        rp = pps.rparams_from_dict(dict(synth.RUN_PARAMS, spacing=0.3))
        nx, ny = pps.pps_run_grid(12.0, 9.0, rp.spacing)
        rout = Guarded(torch, n * pps.RBEST_DTYPE.itemsize)
        sc = Guarded(torch, n * nx * ny * 4)
        pps.pps_run_points(s.ctx, st.data_ptr(), n, rp, rout.ptr, best.ptr,
                           sc.ptr, nx * ny)
        assert rout.intact() and sc.intact()
        torch.cuda.synchronize()
        assert not np.any(sc.body().view(np.float32) == np.frombuffer(
            bytes([CANARY] * 4), np.float32)[0])           # all written
    finally:
        s.close()


def test_proposal_outputs_stay_in_bounds(torch):
    from paper_1909_07717_gb300.proposal import SPEEDS
    n = 3
    batch = synth.PROPOSAL.states(n)
    s = pps.Searcher(max_states=4, max_opp=8)
    net = pps.Net(0, max_batch=4, weights=pps.load_net_weights())
    try:
        st = s.states_to_device(batch)
        pps.pps_net_set_features(net.net, np.asarray(SPEEDS, np.float32),
                                 pps.params_from_dict(synth.DEFAULT_PARAMS))
        fmap = Guarded(torch, n * pps.PPS_NET_H * pps.PPS_NET_W * 4)
        pps.pps_net_forward(net.net, st.data_ptr(), n, fmap.ptr)
        pps.pps_net_sync(net.net)
        assert fmap.intact()
        best = Guarded(torch, n * 32)
        cells = Guarded(torch, n * 100 * 4)
        pps.pps_propose(s.ctx, net.net, st.data_ptr(), n, pps.fine_grid_12x9(),
                        SPEEDS, pps.params_from_dict(synth.DEFAULT_PARAMS), 100,
                        pps.PPS_PROPOSE_FALLBACK, best.ptr, cells.ptr)
        pps.pps_net_sync(net.net)
        assert best.intact() and cells.intact()
    finally:
        net.close()
        s.close()
