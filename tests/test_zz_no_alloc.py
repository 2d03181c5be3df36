"""pps_search_noalloc: the exact search with no device allocation.

Some callers cannot call cudaMalloc: a robot's real-time decision loop that
forbids allocating once it runs, or a process whose device memory is already
owned by another allocator.  pps_search_noalloc serves them with a fixed
scratch array compiled into the library instead of a context.  These tests
call it through the C ABI and check that it returns what the context-based
pps_search returns, on two calls in a row: the second call reuses the array
the first one left behind, so a missed clear would show up as a wrong best
pass.  They also check that a batch above the array's size is refused.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1909_07717_gb300 import build, pps, synth

pytestmark = pytest.mark.gpu

PARAMS = dict(synth.DEFAULT_PARAMS)
SPEEDS = [2.0, 3.5, 5.0, 6.5]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return t


def _with_context(torch, batch, grid, max_opp=8):
    s = pps.Searcher(max_states=batch["ball"].shape[0], max_opp=max_opp)
    try:
        out = s.search(s.states_to_device(batch), batch["ball"].shape[0],
                       grid, SPEEDS, PARAMS)
        torch.cuda.synchronize()
        return (out["best"].cpu().numpy().tobytes(),
                out["mask"].cpu().numpy().view(np.uint32))
    finally:
        s.close()


def _without_allocation(torch, batch, grid, max_opp=8):
    S = batch["ball"].shape[0]
    rec = pps.pack_states(batch)
    states = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    best = torch.empty(S * 32, dtype=torch.uint8, device="cuda")
    mask = torch.empty(S * pps.pps_mask_words(grid, len(SPEEDS)),
                       dtype=torch.int32, device="cuda")
    sp = np.asarray(SPEEDS, np.float32)
    stream = torch.cuda.current_stream().cuda_stream
    pps.pps_search_noalloc(0, stream, max_opp, states.data_ptr(), S, grid,
                           sp.ctypes.data, len(SPEEDS),
                           pps.params_from_dict(PARAMS), best.data_ptr(),
                           mask.data_ptr())
    torch.cuda.synchronize()
    return (best.cpu().numpy().tobytes(),
            mask.cpu().numpy().view(np.uint32))


def _same(ref, got):
    """Both entry points run the same kernel instance on the same inputs:
    the best records and the mask agree byte for byte."""
    assert got[0] == ref[0]
    assert np.array_equal(got[1], ref[1])


def test_noalloc_matches_context_search_two_calls(torch):
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.1)
    # First call: open play without opponents, so every state's best score
    # is high; second call: fewer states, receivers marked, lower scores.
    first = synth.ssl_states(201, 40, K=32, n_opp=0, j_stride=8)
    second = synth.ssl_states(202, 17, K=32, marked=True)
    for batch in (first, second):
        ref = _with_context(torch, batch, grid)
        got = _without_allocation(torch, batch, grid)
        _same(ref, got)
    assert np.all(pps.unpack_best(np.frombuffer(got[0], np.uint8))["status"]
                  == 0)


def test_noalloc_fills_its_whole_array(torch):
    """PPS_NOALLOC_MAX_STATES states, the most one call takes, so the last
    key and count slots of the array are in use, on a coarse grid; then a
    16-slot call (11 opponents) that reuses the first slots."""
    grid = pps.pps_grid_from_field(12.0, 9.0, 1.0)
    n = pps.PPS_NOALLOC_MAX_STATES
    full = synth.ssl_states(203, n, K=8)
    _same(_with_context(torch, full, grid),
          _without_allocation(torch, full, grid))
    eleven = synth.ssl_states(204, 24, K=16, n_opp=11)
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.25)
    _same(_with_context(torch, eleven, grid, max_opp=16),
          _without_allocation(torch, eleven, grid, max_opp=16))


def test_noalloc_rejects_batches_above_its_array(torch):
    grid = pps.pps_grid_from_field(12.0, 9.0, 0.1)
    sp = np.asarray(SPEEDS, np.float32)
    n = pps.PPS_NOALLOC_MAX_STATES + 1
    with pytest.raises(pps.PpsError) as e:
        pps.pps_search_noalloc(0, None, 8, None, n, grid, sp.ctypes.data,
                               len(SPEEDS), None, None, None)
    assert e.value.status == pps.PPS_EINVAL
    assert str(pps.PPS_NOALLOC_MAX_STATES) in pps.pps_last_error(None)
