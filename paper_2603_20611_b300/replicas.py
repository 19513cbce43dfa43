"""Replicas across GPUs: one process per GPU, each holding its own copy of the
Gaussian set and rendering its own random slice batches.

Slices are independent given the Gaussian set (the projection of one slice
reads nothing of another, Eq. 6-10), so the measured step shards with no data
exchange: every rank runs the whole hot path on its own batch and the only
cross-rank step is the reduction of the measurement itself (the slowest rank's
timed seconds and the sum of every rank's evaluations).  A data-parallel fit
would add one sum-reduction of the per-Gaussian gradients per step; that
exchange is not part of this package.
"""
from __future__ import annotations

BATCH_SEED_BASE = 3000
RANK_STRIDE = 7919  # a prime, so no two (rank, step) pairs share a seed for ranks < 7919


def batch_seed(rank: int, step: int) -> int:
    """Seed of the slice batch that `rank` renders at `step` (distinct per rank and step)."""
    if rank < 0 or step < 0 or step >= RANK_STRIDE:
        raise ValueError("rank and step must be non-negative and step < %d" % RANK_STRIDE)
    return BATCH_SEED_BASE + RANK_STRIDE * rank + step


def reduce_timing(seconds: float, evals: float, device=None):
    """(max over ranks of `seconds`, sum over ranks of `evals`).

    Uses the default process group when one is initialised with more than one
    rank (any backend; `device` is where the reduction tensors live: a CUDA
    device under NCCL, None for CPU under gloo); otherwise returns the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(evals)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    e = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())
