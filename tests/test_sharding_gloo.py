"""The multi-GPU path on CPU: world_size-2 gloo ranks build their shards and the job totals
(waveforms summed over ranks, the slowest rank's time). The shards' RNG indices must be
disjoint and cover [0, world * W)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2403_03156_gb300 import sharding
    wl = sharding.rank_workload("plain_fp64_256x128", rank, n_waveforms=16, seed=3, n_steps=10)
    ids = wl["batch"]["wf_ids"]
    gathered = [None] * world
    dist.all_gather_object(gathered, (ids.tolist(), float(wl["batch"]["samples"][:8].sum())))
    W_total, t_max = sharding.job_totals(dist, len(ids), 1.0 + rank)
    out.put((rank, gathered, W_total, t_max))
    dist.destroy_process_group()


def test_shards_disjoint_and_totals_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, W_total, t_max in res:
        assert W_total == 32
        assert t_max == 2.0
        all_ids = np.concatenate([np.asarray(g[0], np.uint64) for g in gathered])
        assert len(set(all_ids.tolist())) == 32
        assert set(all_ids.tolist()) == set(range(32))
        assert gathered[0][1] != gathered[1][1]  # the ranks simulated different data


def test_job_totals_without_process_group():
    from paper_2403_03156_gb300 import sharding
    assert sharding.job_totals(None, 7, 1.5) == (7, 1.5)
