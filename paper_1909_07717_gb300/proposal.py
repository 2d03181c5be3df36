"""The learned proposal path: network, top-k cells, exact refinement.

``Proposal.run`` is one ``pps_propose`` call: the network predicts each
state's 46 x 61 score map, the top-k cells are selected, the exact search
evaluates only the fine (0.025 m) points of those cells, and -- with the
fallback on -- a state whose cells hold no feasible pass is searched on the
full fine grid.  ``Proposal.exact`` runs the plain full-grid search of the
same states, which is both the fallback and the judge of the proposal's
error (``agreement``).
"""
from __future__ import annotations

import numpy as np

from . import pps

# kick speeds of the 12 x 9 m proposal workload (as the batched workload)
SPEEDS = (2.0, 3.5, 5.0, 6.5)
TOPK = 256
REL_TOL = 0.02


class Proposal:
    """A search context and a network sized for ``max_states`` states."""

    def __init__(self, max_states, weights=None, max_opp=8, device=0,
                 stream=None):
        self.searcher = pps.Searcher(max_states, max_opp=max_opp,
                                     device=device, stream=stream)
        if weights is None:
            weights = pps.load_net_weights()
        self.net = pps.Net(device, stream, max_batch=max_states,
                           weights=weights)
        self.torch = self.searcher.torch
        self.grid = pps.fine_grid_12x9()
        self.max_states = max_states

    def set_weights(self, w):
        pps.pps_net_set_weights(self.net.net, w)

    def alloc(self, n, topk=TOPK):
        t = self.torch
        return (t.empty(n * 32, dtype=t.uint8, device=self.searcher.device),
                t.empty((n, topk), dtype=t.int32, device=self.searcher.device))

    def run(self, states_dev, n, speeds=SPEEDS, params=None, topk=TOPK,
            fallback=True, out=None, prune=True):
        """Enqueue the proposal search; returns (best bytes, cells)."""
        best, cells = out if out is not None else self.alloc(n, topk)
        prm = params if isinstance(params, pps.pps_params) else \
            pps.params_from_dict(params)
        pps.pps_propose(self.searcher.ctx, self.net.net,
                        states_dev.data_ptr(), n, self.grid, speeds, prm,
                        topk,
                        (pps.PPS_PROPOSE_FALLBACK if fallback else 0)
                        | (0 if prune else pps.PPS_PROPOSE_NO_PRUNE),
                        best.data_ptr(), cells.data_ptr())
        return best, cells

    def exact(self, states_dev, n, speeds=SPEEDS, params=None, out=None):
        """Enqueue the plain full-grid search; returns the best bytes."""
        o = self.searcher.search(states_dev, n, self.grid, speeds, params,
                                 out=out, mask=False)
        return o["best"]

    def close(self):
        self.net.close()
        self.searcher.close()


def agreement(prop: np.ndarray, exact: np.ndarray, rel=REL_TOL) -> np.ndarray:
    """Per state: the proposal's best score is within ``rel`` of the exact
    one, relative to the exact score's magnitude.  A state with no feasible
    pass agrees when the proposal finds none either.  (The proposal searches
    a subset of the points, so its score never exceeds the exact one.)"""
    pe, ee = prop["idx"] >= 0, exact["idx"] >= 0
    ok = pe == ee
    both = pe & ee
    d = np.abs(prop["score"].astype(np.float64) - exact["score"])
    ok[both] = d[both] <= rel * np.abs(exact["score"][both].astype(np.float64))
    return ok


# The serving workload's proposal: 12 x 9 and 9 x 6 m fields at 0.05 m,
# 6-11 opponents, K = 32, the same four speeds.
SERVING_SPACING = 0.05


class JobsProposal:
    """pps_propose_jobs on a context and network sized for ``max_states``
    states that each carry their own field (grid on the map's lattice)."""

    def __init__(self, max_states, weights, spacing=SERVING_SPACING,
                 max_opp=16, device=0, stream=None):
        self.searcher = pps.Searcher(max_states, max_opp=max_opp,
                                     device=device, stream=stream)
        self.net = pps.Net(device, stream, max_batch=max_states,
                           weights=weights)
        self.torch = self.searcher.torch
        self.spacing = spacing
        self.max_states = max_states

    def jobs_to_device(self, jobs):
        return self.torch.from_numpy(pps.jobs_to_bytes(jobs)).to(
            self.searcher.device)

    def alloc(self, n, topk=TOPK):
        t = self.torch
        return (t.empty(n * 32, dtype=t.uint8, device=self.searcher.device),
                t.empty((n, topk), dtype=t.int32, device=self.searcher.device))

    def run(self, states_dev, jobs_dev, n, speeds=SPEEDS, params=None,
            topk=TOPK, fallback=True, prune=True, out=None):
        """Enqueue the proposal search; returns (best bytes, cells)."""
        best, cells = out if out is not None else self.alloc(n, topk)
        prm = params if isinstance(params, pps.pps_params) else \
            pps.params_from_dict(params)
        pps.pps_propose_jobs(self.searcher.ctx, self.net.net,
                             states_dev.data_ptr(), jobs_dev.data_ptr(), n,
                             self.spacing, len(speeds), prm, topk,
                             (pps.PPS_PROPOSE_FALLBACK if fallback else 0)
                             | (0 if prune else pps.PPS_PROPOSE_NO_PRUNE),
                             best.data_ptr(), cells.data_ptr())
        return best, cells

    def close(self):
        self.net.close()
        self.searcher.close()


def exact_per_field(searcher, batch, spacing=SERVING_SPACING, speeds=SPEEDS,
                    params=None):
    """The plain full-grid search of every state of a batch on its own
    field's grid (one pps_search per field size); host pps_best records."""
    torch = searcher.torch
    S = batch["ball"].shape[0]
    out = np.zeros(S, pps.BEST_DTYPE)
    fields = sorted({(float(a), float(b)) for a, b in
                     zip(batch["field_len"], batch["field_wid"])})
    for L, W in fields:
        idx = np.flatnonzero((batch["field_len"] == L)
                             & (batch["field_wid"] == W))
        sub = {k: np.ascontiguousarray(v[idx]) for k, v in batch.items()}
        grid = pps.pps_grid_from_field(L, W, spacing)
        o = searcher.search(searcher.states_to_device(sub), len(idx), grid,
                            speeds, params, mask=False)
        torch.cuda.synchronize()
        out[idx] = pps.unpack_best(o["best"].cpu().numpy())
    return out
