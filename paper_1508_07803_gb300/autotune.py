"""Launch-shape autotuner for the persistent trace kernel.

The persistent grid's shape -- threads per block and resident blocks per SM
(the number of photon slots in flight per SM) -- and the warp refill
threshold (how many of a warp's 32 lanes must be idle before it takes new
photons: waiting keeps a warp on the same bounce of neighbouring photons,
refilling early keeps lanes busy) trade occupancy, register and shared-memory
pressure and traversal coherence against each other, and the best choice
depends on the optical system (surface count, bounce mix).  The tuners time
the launch on a reduced copy of the work for every candidate and return the
fastest; the results do not depend on the shape (photon-id random streams).
They time the FP32 trace launch alone (accuracy guard off): the guard's FP64
re-trace is a separate launch with its own fixed shape.
"""
from __future__ import annotations

import statistics

from . import RobastError, sources_create, trace, trace_sources

SHAPES = ((64, 0), (128, 0), (256, 0), (128, 2), (128, 3), (256, 1), (64, 4), (64, 6))
REFILL = (8, 16, 24, 32)
TRACE_SHAPES = ((512, 0), (256, 0), (128, 0), (256, 2))


def _time(fn, reps, stream):
    import torch
    fn()  # warm-up (and launch-shape validation)
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def tune_sources(geom, groups, precision: int = 32, max_bounces: int = 100, fraction: float = 0.01,
                 shapes=SHAPES, refill=REFILL, reps: int = 3, seed: int = 0, stream=None):
    """Time trace_sources on `groups` with photon counts scaled by `fraction`
    for every (block, blocks_per_sm, refill_min); returns
    (best (block, blocks_per_sm, refill_min), {candidate: median ms})."""
    import torch
    small = [dict(g, n=max(32, int(g["n"] * fraction))) for g in groups]
    src = sources_create(geom, small)
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream()
    times, last_err = {}, None
    for block, bps in shapes:
        for rm in refill:
            try:
                times[(block, bps, rm)] = _time(
                    lambda: trace_sources(geom, src, counts, seed=seed, precision=precision, max_bounces=max_bounces,
                                          block_size=block, blocks_per_sm=bps, refill_min=rm, stream=stream,
                                          accuracy=False),
                    reps, stream)
            except RobastError as e:
                last_err = e
                continue
    src.close()
    if not times:
        raise RobastError(f"autotune: no candidate launch shape ran ({last_err})")
    best = min(times, key=times.get)
    return best, times


def tune_trace(geom, origins, dirs, wavelengths, precision: int = 32, max_bounces: int = 100, n_sample: int = 2_000_000,
               shapes=TRACE_SHAPES, refill=REFILL, reps: int = 3, seed: int = 0, stream=None, variant_of_photon=None):
    """Time robast.trace on the first n_sample photons (a contiguous slice, as
    the bench's bundles interleave nothing) for every (block, blocks_per_sm,
    refill_min); returns (best, {candidate: median ms})."""
    import torch
    n = min(int(wavelengths.shape[0]), int(n_sample))
    o = origins[:, :n].contiguous()
    d = dirs[:, :n].contiguous()
    w = wavelengths[:n].contiguous()
    v = variant_of_photon[:n].contiguous() if variant_of_photon is not None else None
    if stream is None:
        stream = torch.cuda.current_stream()
    times, last_err = {}, None
    for block, bps in shapes:
        if precision == 64 and block == 512:
            continue
        for rm in refill:
            try:
                times[(block, bps, rm)] = _time(
                    lambda: trace(geom, o, d, w, seed=seed, precision=precision, max_bounces=max_bounces, stream=stream,
                                  block_size=block, blocks_per_sm=bps, refill_min=rm, variant_of_photon=v,
                                  accuracy=False),
                    reps, stream)
            except RobastError as e:
                last_err = e
                continue
    if not times:
        raise RobastError(f"autotune: no candidate launch shape ran ({last_err})")
    best = min(times, key=times.get)
    return best, times
