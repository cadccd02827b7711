"""Batched concentrator study on the GPU: photons generated on the device from
source groups (many cone variants x incidence angles in one launch) against
the oracle fed with its own independently generated photons."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

from parity import compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
robast = pytest.importorskip("paper_1508_07803_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    robast.load()


def _setup(nv=6, angles=(0.0, 12.0, 25.0, 31.0, 40.0), n=301, seed=2):
    scene, groups = W.cone_batch(n_variants=nv, angles_deg=angles, n_per_group=n, seed=seed)
    return scene, groups


@pytest.mark.parametrize("precision", [64, 32])
def test_batched_sources_match_oracle_per_photon(precision):
    scene, groups = _setup()
    geom = robast.build_geometry(scene)
    src = robast.sources_create(geom, groups)
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    out = robast.alloc_outputs(src.n_photons, precision, "cuda")
    robast.trace_sources(geom, src, counts, seed=5, precision=precision, max_bounces=30, out=out,
                         first_photon_id=1000)
    torch.cuda.synchronize()
    g = to_numpy(out)
    b, var, failed = oracle.generate_sources(groups, seed=5, first_photon_id=1000)
    assert failed == 0
    bundle = W.Bundle(b["origins"], b["dirs"], b["wavelengths"])
    if precision == 32:
        bundle = bundle.rounded_to(np.float32)
    ref = oracle.trace(scene, bundle, seed=5, first_photon_id=1000, max_bounces=30, variant_of_photon=var,
                       eps=oracle.default_eps(scene, precision))
    print(compare(g, ref, precision, scene.focal_length, f"sources fp{precision}"))
    # per-group counters agree with the per-photon statuses
    c = counts.cpu().numpy()
    first = 0
    for k, grp in enumerate(groups):
        sl = slice(first, first + grp["n"])
        st = g["status"][sl]
        assert c[k, 7] == grp["n"]
        assert c[k, 0] == g["bounces"][sl].astype(np.int64).sum()
        for s in range(1, 7):
            assert c[k, s] == (st == s).sum()
        first += grp["n"]
    src.close()
    geom.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_batched_sources_order_does_not_change_results(precision):
    """Source mode sorts each chunk of generated photons by origin cell before the trace;
    photon ids, random streams and output slots stay, so the results (FP32 with the guard's
    re-trace, FP64) equal an id-order trace bit for bit."""
    scene, groups = _setup(nv=4, angles=(0.0, 20.0, 35.0), n=20_011)
    geom = robast.build_geometry(scene)
    src = robast.sources_create(geom, groups)
    res = []
    for order in (0, -1):
        counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
        out = robast.alloc_outputs(src.n_photons, precision, "cuda")
        robast.trace_sources(geom, src, counts, seed=3, precision=precision, max_bounces=30, out=out,
                             coherent_order=order)
        torch.cuda.synchronize()
        res.append((counts.cpu().numpy(), to_numpy(out)))
    (c0, o0), (c1, o1) = res
    assert np.array_equal(c0, c1)
    keys = ["status", "bounces", "hit", "dir", "last_surface", "focal_xy"] + (["retraced"] if precision == 32 else [])
    for k in keys:
        assert np.array_equal(o0[k], o1[k]), k
    if precision == 32:
        assert int(o0["retraced"][0]) > 0
    src.close()
    geom.close()


def test_batched_sources_counts_only_and_graph_replay():
    scene, groups = _setup(nv=4, angles=(0.0, 20.0, 35.0), n=20_011)
    geom = robast.build_geometry(scene)
    src = robast.sources_create(geom, groups)
    ref = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    robast.trace_sources(geom, src, ref, seed=9)
    torch.cuda.synchronize()
    # the launch records into a CUDA graph and replays with identical results
    counts = torch.zeros_like(ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        robast.trace_sources(geom, src, counts, seed=9, stream=s)  # warm-up outside capture
        torch.cuda.synchronize()
        counts.zero_()
        with torch.cuda.graph(graph, stream=s):
            robast.trace_sources(geom, src, counts, seed=9, stream=s)
    torch.cuda.synchronize()
    counts.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(counts, 2 * ref)
    ce = (ref[:, 1].double() / ref[:, 7].double()).cpu().numpy()
    assert np.all((ce >= 0) & (ce <= 1))
    src.close()
    geom.close()


def test_batched_sources_reject_bad_groups():
    scene, groups = _setup(nv=2, angles=(0.0,), n=10)
    geom = robast.build_geometry(scene)
    bad = dict(groups[0])
    bad["variant"] = 7
    with pytest.raises(robast.RobastError, match="variant"):
        robast.sources_create(geom, [bad])
    bad = dict(groups[0])
    bad["dir"] = (0.0, 0.0, -2.0)
    with pytest.raises(robast.RobastError, match="unit"):
        robast.sources_create(geom, [bad])
    geom.close()


def test_tolerance_sweep_r80_distribution_matches_oracle():
    """Tilt-error realisations as variants of one launch; the spot-diagram
    R80 of every realisation agrees with the oracle's to 0.1%, and larger
    errors give larger spots."""
    from oracle import metrics
    nr, m = 6, 3_001
    scene, b, vop = W.tolerance_sweep(n_realizations=nr, tilt_sigma=1e-3, photons_per_realization=m, seed=3)
    geom = robast.build_geometry(scene)
    o = torch.from_numpy(b.origins).to("cuda", torch.float32)
    d = torch.from_numpy(b.dirs).to("cuda", torch.float32)
    w = torch.from_numpy(b.wavelengths).to("cuda", torch.float32)
    out = robast.trace(geom, o, d, w, seed=5, variant_of_photon=torch.from_numpy(vop).cuda())
    res = robast.psf(geom, out["status"], out["focal_xy"], windows=[(v * m, m) for v in range(nr)])
    ref = oracle.trace(scene, b.rounded_to(np.float32), seed=5, variant_of_photon=vop,
                       eps=oracle.default_eps(scene, 32))
    r80 = []
    for v, (n_det, cx, cy, r) in enumerate(res):
        sl = slice(v * m, (v + 1) * m)
        want = metrics.psf(ref["status"][sl], ref["focal_xy"][:, sl])
        assert n_det == want["n_detected"]
        assert r == pytest.approx(want["r80"], rel=1e-3)
        r80.append(r)
    # realisations differ (independent tilt errors)
    assert np.std(r80) > 0
    geom.close()
    scene0, b0, vop0 = W.tolerance_sweep(n_realizations=2, tilt_sigma=0.0, photons_per_realization=m, seed=3)
    g0 = robast.build_geometry(scene0)
    o0 = torch.from_numpy(b0.origins).to("cuda", torch.float32)
    d0 = torch.from_numpy(b0.dirs).to("cuda", torch.float32)
    w0 = torch.from_numpy(b0.wavelengths).to("cuda", torch.float32)
    out0 = robast.trace(g0, o0, d0, w0, seed=5, variant_of_photon=torch.from_numpy(vop0).cuda())
    r0 = robast.psf(g0, out0["status"], out0["focal_xy"], windows=[(0, m)])[0][3]
    assert r0 < np.mean(r80)
    g0.close()


def test_autotuners_pick_a_candidate_and_results_do_not_depend_on_it():
    """The launch-shape tuners time every (block, blocks per SM, refill threshold)
    candidate and return the fastest; tracing with it gives the same results as the
    default launch (photon-id random streams)."""
    from paper_1508_07803_gb300 import autotune
    scene, groups = _setup(nv=2, angles=(0.0, 30.0), n=20_000)
    geom = robast.build_geometry(scene)
    best, table = autotune.tune_sources(geom, groups, max_bounces=30, fraction=0.05,
                                        shapes=((128, 0), (64, 2)), refill=(8, 24))
    assert best in table and len(table) == 4 and all(t > 0 for t in table.values())
    src = robast.sources_create(geom, groups)
    a = torch.zeros((src.n_groups, 8), dtype=torch.int64, device="cuda")
    b = torch.zeros_like(a)
    robast.trace_sources(geom, src, a, seed=3, max_bounces=30)
    robast.trace_sources(geom, src, b, seed=3, max_bounces=30, block_size=best[0], blocks_per_sm=best[1],
                         refill_min=best[2])
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    src.close()
    geom.close()
    scene, bun = W.lst_workload(40_000, seed=4, angles_deg=(1.0,))
    geom = robast.build_geometry(scene)
    o = torch.from_numpy(bun.origins).to("cuda", torch.float32)
    d = torch.from_numpy(bun.dirs).to("cuda", torch.float32)
    w = torch.from_numpy(bun.wavelengths).to("cuda", torch.float32)
    best, table = autotune.tune_trace(geom, o, d, w, n_sample=20_000, shapes=((512, 0), (128, 0)), refill=(16, 24))
    assert best in table and len(table) == 4
    ref = to_numpy(robast.trace(geom, o, d, w, seed=2))
    got = to_numpy(robast.trace(geom, o, d, w, seed=2, block_size=best[0], blocks_per_sm=best[1], refill_min=best[2]))
    for k in ("status", "bounces", "hit", "dir", "last_surface", "focal_xy"):
        assert np.array_equal(ref[k], got[k]), k
    geom.close()
