"""Train the proposal network on exact labels, on the GPU.

Labels: the exact search (``pps_search``) of every training state on the
0.025 m grid of the 12 x 9 m field writes each point's best score over the
kick speeds; ``pps_net_labels`` reduces those to the 46 x 61 map -- per map
pixel, the best score of the 8 x 8 fine points centred on it, with cells
that hold no feasible pass set to the floor -1.2 (below any score the value
function gives: the angle term is >= 0, the distance term >= -1.1 on a
12 x 9 m field, the margin >= 0).  Training: Adam on the top-focused mean
squared error (``pps_net_set_loss``: full weight for the pixels whose label
or prediction comes within --top-band of the state's best label,
--low-weight for the rest, --under-weight times more where the prediction
is below the label), a cosine learning-rate decay, every step a
``pps_net_train_step`` (the library's own forward and backward kernels).
The whole training set -- state records and label maps -- stays resident in
device memory (1M states: 0.3 GB of records, 11 GB of labels).

    python -m paper_1909_07717_gb300.train_proposal --states 1048576 \\
        --epochs 4 --out paper_1909_07717_gb300/weights/proposal_12x9_v4_K64_J8.bin
    python -m paper_1909_07717_gb300.train_proposal --workload serving \\
        --states 1048576 --epochs 4

Prints one JSON line with the label and training times, the losses and the
held-out agreement of the proposal (top-256, fallback off and on) with the
plain search.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import pps, synth
from .proposal import SPEEDS, TOPK, Proposal, agreement

LABEL_FLOOR = -1.2
CHUNK = 4096
TRAIN_SEED = 100_000      # chunk c of the training set: seed TRAIN_SEED + c
HELDOUT_SEED = 7          # held-out states (never trained on)


SERVING_SEED0 = 300_000   # training chunks of the serving workload
SERVING_HELDOUT_SEED = 9


def make_serving_labels(torch, searcher, net, n_states, seed0, chunk=CHUNK):
    """States of the serving workload (synth.serving_states: 12 x 9 and
    9 x 6 m fields, 6-11 opponents, K = 32) and their label maps from the
    exact search on each field's 0.05 m grid (pps_net_labels_grid: the best
    of each map pixel's 4 x 4 fine points, the floor where the pixel holds
    no point of the field)."""
    from .proposal import SERVING_SPACING
    dev = searcher.device
    rs = pps.STATE_DTYPE.itemsize
    rec = torch.empty(n_states * rs, dtype=torch.uint8, device=dev)
    labels = torch.empty((n_states, pps.PPS_NET_H, pps.PPS_NET_W),
                         dtype=torch.float32, device=dev)
    grids = {f: pps.pps_grid_from_field(f[0], f[1], SERVING_SPACING)
             for f in ((12.0, 9.0), (9.0, 6.0))}
    Pmax = max(g.nx * g.ny for g in grids.values())
    pb = torch.empty((chunk, Pmax), dtype=torch.float32, device=dev)
    lab = torch.empty((chunk, pps.PPS_NET_H, pps.PPS_NET_W),
                      dtype=torch.float32, device=dev)
    for c in range(0, n_states, chunk):
        n = min(chunk, n_states - c)
        batch = synth.serving_states(seed0 + c // chunk, n)
        host = torch.from_numpy(pps.pack_states(batch).view(np.uint8).copy())
        rec[c * rs:(c + n) * rs].copy_(host)
        for f, grid in grids.items():
            idx = np.flatnonzero((batch["field_len"] == f[0])
                                 & (batch["field_wid"] == f[1]))
            if not len(idx):
                continue
            sub = synth.take(batch, idx)
            P = grid.nx * grid.ny
            pbv = pb.view(-1)[:len(idx) * P].view(len(idx), P)
            out = searcher.alloc_outputs(len(idx), grid, len(SPEEDS),
                                         mask=False)
            searcher.search(searcher.states_to_device(sub), len(idx), grid,
                            SPEEDS, synth.DEFAULT_PARAMS, out=out, mask=False,
                            point_best=pbv)
            pps.pps_net_labels_grid(net.net, pbv.data_ptr(), len(idx), grid,
                                    LABEL_FLOOR, lab.data_ptr())
            ti = torch.from_numpy(idx + c).to(dev)
            labels.index_copy_(0, ti, lab[:len(idx)])
    torch.cuda.synchronize()
    return rec, labels


def evaluate_serving(torch, weights, n_states=4096,
                     seed=SERVING_HELDOUT_SEED):
    """Held-out agreement of the per-job proposal with the plain search on
    the serving workload, overall and per field."""
    from .proposal import JobsProposal, exact_per_field
    batch = synth.serving_states(seed, n_states)
    pr = JobsProposal(n_states, weights)
    try:
        st = pr.searcher.states_to_device(batch)
        jobs = pr.jobs_to_device(pps.field_jobs(batch, pr.spacing, SPEEDS))
        ex = exact_per_field(pr.searcher, batch, pr.spacing, SPEEDS,
                             synth.DEFAULT_PARAMS)
        res = {}
        for fb in (False, True):
            b, _ = pr.run(st, jobs, n_states, fallback=fb)
            res[fb] = pps.unpack_best(b.cpu().numpy())
    finally:
        pr.close()
    big = batch["field_len"] == 12.0
    ok = agreement(res[False], ex)
    return {"states": n_states,
            "agree_no_fallback": float(ok.mean()),
            "agree_12x9": float(ok[big].mean()),
            "agree_9x6": float(ok[~big].mean()),
            "agree_fallback": float(agreement(res[True], ex).mean()),
            "fallback_states": int(((res[False]["idx"] == -1)
                                    & (ex["idx"] >= 0)).sum())}


def make_labels(torch, searcher, net, n_states, seed0, chunk=CHUNK):
    """States and exact label maps of n_states training states, resident
    on the device: (uint8 records, float32 labels n x 46 x 61)."""
    dev = searcher.device
    rec = torch.empty(n_states * pps.STATE_DTYPE.itemsize, dtype=torch.uint8,
                      device=dev)
    labels = torch.empty((n_states, pps.PPS_NET_H, pps.PPS_NET_W),
                         dtype=torch.float32, device=dev)
    grid = pps.fine_grid_12x9()
    P = grid.nx * grid.ny
    pb = torch.empty((chunk, P), dtype=torch.float32, device=dev)
    out = searcher.alloc_outputs(chunk, grid, len(SPEEDS), mask=False)
    rs = pps.STATE_DTYPE.itemsize
    for c in range(0, n_states, chunk):
        n = min(chunk, n_states - c)
        batch = synth.ssl_states(seed0 + c // chunk, n, K=64)
        host = torch.from_numpy(pps.pack_states(batch).view(np.uint8).copy())
        part = rec[c * rs:(c + n) * rs]
        part.copy_(host)
        searcher.search(part, n, grid, SPEEDS, synth.DEFAULT_PARAMS, out=out,
                        mask=False, point_best=pb)
        pps.pps_net_labels(net.net, pb.data_ptr(), n, LABEL_FLOOR,
                           labels[c:c + n].data_ptr())
    torch.cuda.synchronize()
    return rec, labels


def train(net, rec, labels, n_states, batch, epochs, lr0, seed=0, log=None):
    rs = pps.STATE_DTYPE.itemsize
    nb = n_states // batch
    total = epochs * nb
    rng = np.random.default_rng(seed)
    step, losses = 0, []
    base_r, base_l = rec.data_ptr(), labels.data_ptr()
    lab_bytes = pps.PPS_NET_H * pps.PPS_NET_W * 4
    for ep in range(epochs):
        for b in rng.permutation(nb):
            warm = min(1.0, (step + 1) / 200)
            lr = lr0 * warm * 0.5 * (1 + math.cos(math.pi * step / total))
            want = step % 250 == 0 or step == total - 1
            loss = pps.pps_net_train_step(
                net.net, base_r + int(b) * batch * rs,
                base_l + int(b) * batch * lab_bytes, batch, max(lr, 1e-6),
                want_loss=want)
            if want:
                losses.append((step, loss))
                if log:
                    log(f"step {step}/{total} epoch {ep} loss {loss:.5f}")
            step += 1
    return losses


def evaluate(torch, weights, n_states=4096, seed=HELDOUT_SEED):
    batch = synth.ssl_states(seed, n_states, K=64)
    pr = Proposal(n_states, weights)
    try:
        st = pr.searcher.states_to_device(batch)
        ex = pps.unpack_best(pr.exact(st, n_states).cpu().numpy())
        nofb, _ = pr.run(st, n_states, fallback=False)
        nofb = pps.unpack_best(nofb.cpu().numpy())
        fb, _ = pr.run(st, n_states, fallback=True)
        fb = pps.unpack_best(fb.cpu().numpy())
    finally:
        pr.close()
    return {"states": n_states,
            "agree_no_fallback": float(agreement(nofb, ex).mean()),
            "agree_fallback": float(agreement(fb, ex).mean()),
            "fallback_states": int(((nofb["idx"] == -1)
                                    & (ex["idx"] >= 0)).sum())}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--states", type=int, default=1 << 20)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--top-band", type=float, default=0.5)
    ap.add_argument("--low-weight", type=float, default=0.05)
    ap.add_argument("--under-weight", type=float, default=8.0)
    ap.add_argument("--heldout", type=int, default=4096)
    ap.add_argument("--workload", choices=["fine_12x9", "serving"],
                    default="fine_12x9",
                    help="fine_12x9: 12 x 9 m, 8 v 8, K 64, 0.025 m grid; "
                         "serving: 12 x 9 / 9 x 6 m, 6-11 opponents, K 32, "
                         "0.05 m grids")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    serving = args.workload == "serving"
    if args.out is None:
        args.out = pps.SERVING_WEIGHTS if serving else pps.PROPOSAL_WEIGHTS

    import torch
    from . import build
    build.build()
    t0 = time.time()
    searcher = pps.Searcher(CHUNK, max_opp=16 if serving else 8)
    net = pps.Net(max_batch=max(args.batch, CHUNK),
                  weights=pps.init_weights(args.init_seed, zero_output=True))
    pps.pps_net_set_loss(net.net, args.top_band, args.low_weight,
                         args.under_weight)
    if serving:
        rec, labels = make_serving_labels(torch, searcher, net, args.states,
                                          SERVING_SEED0)
    else:
        rec, labels = make_labels(torch, searcher, net, args.states,
                                  TRAIN_SEED)
    searcher.close()
    t_label = time.time() - t0
    t1 = time.time()
    losses = train(net, rec, labels, args.states, args.batch, args.epochs,
                   args.lr, log=lambda m: print(m, flush=True))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    w = pps.pps_net_get_weights(net.net)
    net.close()
    del rec, labels
    pps.save_net_weights(args.out, w)
    ev_fn = evaluate_serving if serving else evaluate
    ev = ev_fn(torch, w, args.heldout)
    # zero weights: the network adds nothing to the coarse-score channel
    ev_feat = ev_fn(torch, np.zeros(pps.PPS_NET_PARAMS, np.float32),
                    args.heldout)
    print(json.dumps({"workload": args.workload,
                      "states": args.states, "epochs": args.epochs,
                      "batch": args.batch, "lr": args.lr,
                      "top_band": args.top_band,
                      "low_weight": args.low_weight,
                      "under_weight": args.under_weight,
                      "label_s": round(t_label, 2),
                      "train_s": round(t_train, 2),
                      "first_loss": losses[0][1], "last_loss": losses[-1][1],
                      "heldout": ev, "heldout_features_only": ev_feat,
                      "topk": TOPK, "out": args.out}))


if __name__ == "__main__":
    main()
