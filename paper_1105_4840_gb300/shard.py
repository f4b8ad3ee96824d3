"""Host side of a PPP run sharded over processes (one GPU each).

Every (window, replica) simulation is independent (Sec. III (ii)), so a
shard runs every window with its own block of replicas: shard `rank` uses
replica uids uid_base + w * R + r with uid_base = rank * s * R, disjoint from
every other shard's.  The only exchange is the per-replica partial sums of
the reductions (pmf_run_partials, [s][R][5] doubles per shard); gathering them
and concatenating along the replica axis gives the partials of the union of
the replicas, which pmf_free_energy_from_partials turns into the estimates.
"""
from __future__ import annotations

import numpy as np


def shard_uid_base(rank: int, n_windows: int, replicas: int) -> int:
    """First replica uid of shard `rank` (each shard: n_windows x replicas)."""
    if rank < 0 or n_windows < 1 or replicas < 1:
        raise ValueError("rank >= 0, n_windows >= 1, replicas >= 1")
    base = rank * n_windows * replicas
    if base + n_windows * replicas > 2 ** 32:
        raise ValueError("replica uids exceed 32 bits")
    return base


def merge_partials(parts) -> np.ndarray:
    """Concatenate shards' partials [s][R_k][5] along the replica axis."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    s = parts[0].shape[0]
    if any(p.ndim != 3 or p.shape[0] != s or p.shape[2] != 5 for p in parts):
        raise ValueError("partials must be [n_windows][replicas][5] with equal n_windows")
    return np.concatenate(parts, axis=1)


def gather_partials(local, group=None, device=None) -> np.ndarray:
    """All-gather every rank's partials (equal shapes) with torch.distributed
    and merge them in rank order; `device` is where the collective runs
    (CPU tensors for gloo, a CUDA device for nccl)."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64), device=device)
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    return merge_partials([b.cpu().numpy() for b in bufs])
