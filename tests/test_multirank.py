"""The sharded multi-GPU path's host logic on two gloo ranks (CPU).

Each rank draws its own states (rank-derived seed), the ranks agree on the
slowest rank's time through one max reduction, and the job rate counts
every rank's work over that time.  No GPU is involved.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    from paper_1909_07717_gb300 import shard, synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    try:
        w = synth.BATCHED
        seed = shard.rank_seed(w.seed, rank)
        batch = synth.ssl_states(seed, 16, K=w.K)
        digest = torch.tensor([float(np.sum(batch["ball"].astype(np.float64)))],
                              dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, digest)
        local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
        slowest = shard.max_over_ranks(local_ms, dist)
        rate = shard.job_rate(100, world, 5, slowest)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([seed, slowest, rate]
                         + [g.item() for g in gathered]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
             join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == 1 and r1[0] == 1001          # distinct seeds
    assert r0[3] != r0[4]                        # distinct states
    assert np.array_equal(r0[3:], r1[3:])        # both saw both digests
    assert r0[1] == r1[1] == 20.0                # max over ranks
    assert r0[2] == r1[2] == pytest.approx(2 * 100 * 5 / 0.020)


def test_single_rank_is_identity():
    from paper_1909_07717_gb300 import shard
    assert shard.max_over_ranks(12.5) == 12.5
    assert shard.rank_seed(1, 0) == 1
    assert shard.job_rate(10, 1, 2, 1000.0) == 20.0
