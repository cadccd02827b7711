"""Multi-GPU host logic: photon-id sharding and the reductions of the timed run.

Photons are independent and every photon's random stream is keyed by its id
(robast_trace_opts.first_photon_id), so ranks need no collective in the data
path: each rank traces its own contiguous id range, and the union of the
ranks' results is exactly what one GPU tracing all ids produces.  Only the
timing (max over ranks) and the counters (sums) cross ranks.
"""
from __future__ import annotations


def shard(n_total: int, rank: int, world: int):
    """Contiguous, disjoint photon range of `rank`: (first id, count); the ranges cover [0, n_total)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    lo = n_total * rank // world
    hi = n_total * (rank + 1) // world
    return lo, hi - lo


def replica_first_id(rank: int, n_per_rank: int) -> int:
    """Weak scaling: every rank traces a full workload of n_per_rank photons
    with its own id range [rank n, (rank + 1) n)."""
    return rank * n_per_rank


def all_reduce_scalar(x: float, op: str = "max", device=None) -> float:
    """Max or sum of a float over the ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
