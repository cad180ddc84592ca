"""Weak-scaling shards of a workload over ranks (one process per GPU).

The chains are independent (Sec. 2.4 batches them with no interaction), so a multi-GPU job is
one shard of waveforms per rank with no data-path collective: each rank simulates its own
shard with its own seed, and the shards' RNG indices (wf_ids) are disjoint, so no two chains
of the job share a Philox stream. The only exchange is the end-of-run totals: the waveforms
summed over ranks and the slowest rank's time."""
from __future__ import annotations

import numpy as np


def rank_workload(name: str, rank: int, n_waveforms=None, seed: int = 0, n_steps=None):
    """Rank `rank`'s shard of the named workload: seed + 1000 rank, waveform ids rank * W + i."""
    from . import workloads
    wl = workloads.make_workload(name, n_waveforms=n_waveforms, seed=seed + 1000 * rank, n_steps=n_steps)
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    b["wf_ids"] = np.arange(W, dtype=np.uint64) + np.uint64(rank * W)
    return wl


def job_totals(dist, n_local: int, elapsed_s: float, device=None):
    """(waveforms over all ranks, the slowest rank's elapsed time) by two all-reduces; without
    an initialised process group, the local values."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return int(n_local), float(elapsed_s)
    import torch
    t = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    e = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.MAX)
    return int(t.item()), float(e.item())
