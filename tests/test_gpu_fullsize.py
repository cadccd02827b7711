"""Full-size launches (the sizes and launch configuration bench.py times)
checked on sampled photons the oracle traces one by one.

The dish workload (5 x 1e7 photons), the two-mirror workload (8 x 1e7, FP32 and FP64) and
the GCT-like workload (5 x 1e7) are traced whole on the GPU with the default launch (persistent grid, coherent
order, FP32 accuracy guard); windows of contiguous photon ids at random
offsets, 1e6 photons per workload in all, are traced by the oracle with
first_photon_id set to the window start and compared photon by photon with
the same fixed tolerances as the small cases: at 1e6 photons the FP32 status
criterion (at least 99.999% identical) allows 10 mismatches, all at edges.
The batched concentrator study (64 variants x 41 angles x 2e6 photons, ids
beyond 2^32) is checked through invariants of its per-group counters and by
re-tracing 1e6 of its photons, in windows of several groups, at their
original ids.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

from parity import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
robast = pytest.importorskip("paper_1508_07803_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    robast.load()


def _windows(n, k, size, seed):
    rng = np.random.default_rng(seed)
    starts = np.sort(rng.choice(n - size, size=k, replace=False))
    return [(int(s), size) for s in starts]


def _check_windows(scene, b, out, precision, seed, wins, max_bounces=100):
    g = {k: v for k, v in out.items() if k not in ("counters", "retraced")}
    for s0, c in wins:
        sl = slice(s0, s0 + c)
        part = W.Bundle(np.ascontiguousarray(b.origins[:, sl]), np.ascontiguousarray(b.dirs[:, sl]),
                        b.wavelengths[sl].copy())
        if precision == 32:
            part = part.rounded_to(np.float32)
        ref = oracle.trace(scene, part, seed=seed, first_photon_id=s0, max_bounces=max_bounces,
                           eps=oracle.default_eps(scene, precision))
        got = {}
        for k, v in g.items():
            t = v[..., s0:s0 + c]
            got[k] = t.cpu().numpy()
        compare(got, ref, precision, scene.focal_length, f"window {s0}")


@pytest.mark.parametrize("precision", [32, 64])
def test_dish_full_size_sampled(precision):
    npa = 10_000_000
    scene, b = W.lst_workload(npa, seed=0)
    geom = robast.build_geometry(scene)
    dt = torch.float32 if precision == 32 else torch.float64
    o = torch.from_numpy(b.origins).to("cuda", dt)
    d = torch.from_numpy(b.dirs).to("cuda", dt)
    w = torch.from_numpy(b.wavelengths).to("cuda", dt)
    out = robast.trace(geom, o, d, w, seed=0, precision=precision)
    torch.cuda.synchronize()
    c = out["counters"].cpu().numpy()
    assert c[7] == b.n and c[1:7].sum() == b.n
    if precision == 32:
        assert int(out["retraced"][1]) == 0  # every photon over the guard's bounds was re-traced
    _check_windows(scene, b, out, precision, 0, _windows(b.n, 10, 100_000, seed=precision))
    geom.close()


def _full_size(scene, b, precision, seed, win_seed):
    geom = robast.build_geometry(scene)
    dt = torch.float32 if precision == 32 else torch.float64
    o = torch.from_numpy(b.origins).to("cuda", dt)
    d = torch.from_numpy(b.dirs).to("cuda", dt)
    w = torch.from_numpy(b.wavelengths).to("cuda", dt)
    out = robast.trace(geom, o, d, w, seed=seed, precision=precision)
    torch.cuda.synchronize()
    c = out["counters"].cpu().numpy()
    assert c[7] == b.n and c[1:7].sum() == b.n
    if precision == 32:
        assert int(out["retraced"][1]) == 0
    _check_windows(scene, b, out, precision, seed, _windows(b.n, 10, 100_000, seed=win_seed))
    geom.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_two_mirror_full_size_sampled(precision):
    """The SCT-like workload the bench times (8 field angles x 1e7 photons)."""
    scene, b = W.sct_workload(10_000_000, seed=0)
    _full_size(scene, b, precision, 1, 7 + precision)


def test_gct_full_size_sampled():
    """The GCT-like workload the bench times (5 field angles x 1e7 photons), FP32 with the guard."""
    scene, b = W.gct_workload(10_000_000, seed=0)
    _full_size(scene, b, 32, 2, 11)


def test_batched_full_size_counters_and_sampled_ids():
    scene, groups = W.cone_batch(n_variants=64, angles_deg=W.CONE_ANGLES_DEG, n_per_group=2_000_000, seed=0)
    geom = robast.build_geometry(scene)
    src = robast.sources_create(geom, groups)
    assert src.n_photons == 64 * 41 * 2_000_000 > 2**32
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    retraced = torch.zeros(2, dtype=torch.int64, device="cuda")
    robast.trace_sources(geom, src, counts, seed=0, precision=32, max_bounces=30, out={"retraced": retraced})
    torch.cuda.synchronize()
    # launched in chunks of the re-trace queue's size: every photon over the bounds was re-traced
    assert int(retraced[1]) == 0 and int(retraced[0]) > 0
    c = counts.cpu().numpy()
    assert np.all(c[:, 7] == 2_000_000)
    assert np.all(c[:, 1:7].sum(axis=1) == c[:, 7])
    assert np.all(c[:, 6] == 0)  # no ERROR photons
    assert np.all(c[:, 0] >= c[:, 1])  # a detected photon made at least one interaction
    ce = (c[:, 1] / c[:, 7]).reshape(64, 41)
    assert np.all(ce[:, :20].mean(axis=1) > ce[:, 35:].mean(axis=1))  # cutoff at large incidence
    # windows of single groups re-traced at their original photon ids (beyond 2^32 included):
    # 8 windows of 125k photons, 1e6 in all
    first = np.cumsum([0] + [g["n"] for g in groups])
    rng = np.random.default_rng(3)
    m = 125_000
    for gi in rng.choice(len(groups), size=7, replace=False).tolist() + [len(groups) - 1]:
        j = int(rng.integers(0, groups[gi]["n"] - m))
        pid0 = int(first[gi]) + j
        one = [dict(groups[gi], n=m)]
        s1 = robast.sources_create(geom, one)
        cnt1 = torch.zeros((1, 8), dtype=torch.int64, device="cuda")
        out = robast.alloc_outputs(m, 32, "cuda")
        robast.trace_sources(geom, s1, cnt1, seed=0, precision=32, max_bounces=30, out=out, first_photon_id=pid0)
        torch.cuda.synchronize()
        bb, var, failed = oracle.generate_sources(one, seed=0, first_photon_id=pid0)
        assert failed == 0
        bundle = W.Bundle(bb["origins"], bb["dirs"], bb["wavelengths"]).rounded_to(np.float32)
        ref = oracle.trace(scene, bundle, seed=0, first_photon_id=pid0, max_bounces=30, variant_of_photon=var,
                           eps=oracle.default_eps(scene, 32))
        assert int(out["retraced"][1]) == 0
        compare({k: v.cpu().numpy() for k, v in out.items() if k not in ("counters", "retraced")}, ref, 32,
                scene.focal_length, f"group {gi} ids {pid0}..")
        s1.close()
    src.close()
    geom.close()
