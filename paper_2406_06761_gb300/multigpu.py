"""Placement of Wally's server work over several GPUs (one process per GPU).

Queries are independent (the paper evaluates each on its own core with no
inter-query synchronisation, Sec. 8), so GPUs share no state on the data path.
Two placements:

- replicas: every rank holds the whole encoded database and takes its own
  slice of the query stream (or, for the weak-scaling benchmark, its own
  copy of a batch);
- cluster shards: every rank holds a subset of the clusters, chosen to
  balance chunks x expected queries, and the host routes each query to the
  rank that owns its cluster (harness.DeviceWorkload(shard=...) builds a
  rank's share; bench.py uses it under torchrun).

Only timing crosses ranks: a barrier and the maximum of the step times.
"""
from __future__ import annotations

import numpy as np


def split_stream(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous slice [lo, hi) of n queries for `rank` (replicas)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_clusters(chunks, expected_queries, world: int) -> np.ndarray:
    """Owner rank of every cluster: longest-processing-time-first greedy on
    load = chunks x (expected queries + 1), so that every rank gets clusters
    and the heaviest rank stays within one cluster of the average."""
    chunks = np.asarray(chunks, dtype=np.float64)
    load = chunks * (np.asarray(expected_queries, dtype=np.float64) + 1.0)
    owner = np.empty(len(load), dtype=np.int64)
    acc = np.zeros(world)
    for c in np.argsort(-load, kind="stable"):
        r = int(np.argmin(acc))
        owner[c] = r
        acc[r] += load[c]
    return owner


def local_clusters(owner: np.ndarray, rank: int) -> np.ndarray:
    """Global ids of the clusters `rank` owns, in id order (its local order)."""
    return np.flatnonzero(owner == rank)


def route(ids, owner: np.ndarray, rank: int) -> tuple[np.ndarray, np.ndarray]:
    """Queries of `rank` under cluster sharding: (query indices, local cluster ids)."""
    ids = np.asarray(ids)
    mine = np.flatnonzero(owner[ids] == rank)
    local_of = -np.ones(len(owner), dtype=np.int64)
    lc = local_clusters(owner, rank)
    local_of[lc] = np.arange(len(lc))
    return mine, local_of[ids[mine]].astype(np.uint32)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
