"""Launch-shape autotuner for the persistent trace kernel.

The persistent grid's shape -- threads per block and resident blocks per SM
(the number of photon slots in flight per SM) -- trades occupancy against
register and shared-memory pressure, and the best choice depends on the
optical system (surface count, bounce mix).  tune_sources() times the batched
source launch on a reduced copy of the groups for every candidate shape and
returns the fastest; the result is used for the full launch.
"""
from __future__ import annotations

import statistics

from . import RobastError, sources_create, trace_sources

CANDIDATES = ((64, 0), (128, 0), (256, 0), (128, 2), (128, 3), (256, 1), (64, 4), (64, 6))


def tune_sources(geom, groups, precision: int = 32, max_bounces: int = 100, fraction: float = 0.01,
                 candidates=CANDIDATES, reps: int = 3, seed: int = 0, stream=None):
    """Time trace_sources on `groups` with photon counts scaled by `fraction`;
    returns (best (block, blocks_per_sm), {shape: median ms})."""
    import torch
    small = [dict(g, n=max(32, int(g["n"] * fraction))) for g in groups]
    src = sources_create(geom, small)
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream()
    times = {}
    for block, bps in candidates:
        try:
            trace_sources(geom, src, counts, seed=seed, precision=precision, max_bounces=max_bounces,
                          block_size=block, blocks_per_sm=bps, stream=stream)
        except RobastError:
            continue
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            trace_sources(geom, src, counts, seed=seed, precision=precision, max_bounces=max_bounces,
                          block_size=block, blocks_per_sm=bps, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        times[(block, bps)] = statistics.median(ms)
    src.close()
    if not times:
        raise RobastError("autotune: no candidate launch shape ran")
    best = min(times, key=times.get)
    return best, times
