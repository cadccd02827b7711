"""The allocation-free spot-diagram entry point (robast_psf_noalloc).

Some callers cannot allocate device memory when they need these statistics
(a caching allocator that owns the device, a fixed memory budget);
robast_psf_noalloc serves them from a fixed scratch array inside the library.
(It synchronises its stream between rounds, so it is not for streams that are
being captured into a CUDA graph.)  This test calls it through the C ABI and checks it against the
allocating entry point robast_psf on two calls in a row (different traces,
window layouts and precisions), since the scratch keeps the previous call's
contents.  The file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

robast = pytest.importorskip("paper_1508_07803_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    robast.load()


def _trace(precision, npa, seed, angles):
    scene, b = W.lst_workload(npa, seed=seed, angles_deg=angles)
    geom = robast.build_geometry(scene)
    dt = torch.float32 if precision == 32 else torch.float64
    o = torch.from_numpy(b.origins).to("cuda", dt)
    d = torch.from_numpy(b.dirs).to("cuda", dt)
    w = torch.from_numpy(b.wavelengths).to("cuda", dt)
    out = robast.trace(geom, o, d, w, seed=seed, precision=precision)
    return geom, out


def _same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        if math.isnan(y):
            assert math.isnan(x)
        else:
            assert x == pytest.approx(y, rel=1e-12, abs=1e-15)


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    # call 1: FP32, five field angles of 40k photons (bins above the cap force refinement)
    npa = 40_000
    geom, out = _trace(32, npa, seed=21, angles=W.LST_ANGLES_DEG)
    wins = [(k * npa, npa) for k in range(5)]
    ref = robast.psf(geom, out["status"], out["focal_xy"], precision=32, windows=wins)
    got = robast.psf_noalloc(out["status"], out["focal_xy"], wins, precision=32)
    for a, b in zip(got, ref):
        _same(a, b)
    # call 2: FP64, other windows incl. a one-photon window and a whole-range window
    npa2 = 9_001
    geom2, out2 = _trace(64, npa2, seed=22, angles=(0.5, 2.0))
    wins2 = [(0, npa2), (npa2, npa2), (0, 2 * npa2), (17, 1)]
    ref2 = robast.psf(geom2, out2["status"], out2["focal_xy"], precision=64, windows=wins2)
    got2 = robast.psf_noalloc(out2["status"], out2["focal_xy"], wins2, precision=64)
    for a, b in zip(got2, ref2):
        _same(a, b)
    # and the first case again, after the scratch held the second call's contents
    again = robast.psf_noalloc(out["status"], out["focal_xy"], wins, precision=32)
    for a, b in zip(again, ref):
        _same(a, b)
    geom.close()
    geom2.close()


def test_noalloc_rejects_too_many_windows():
    geom, out = _trace(32, 1_000, seed=3, angles=(0.0,))
    with pytest.raises(robast.RobastError, match="n_windows"):
        robast.psf_noalloc(out["status"], out["focal_xy"], [(0, 10)] * 65)
    geom.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_refines_crowded_bins(precision):
    """A ring of 160k photons at one radius holds the 80% rank: the first
    histogram bin is far over the selection cap, so the bounded-scratch
    entry point must refine it; both entry points and a plain numpy
    nearest-rank agree."""
    rng = np.random.default_rng(5)
    a = 0.02
    inner = rng.uniform(0, a / 2, 40_000), rng.uniform(0, 2 * np.pi, 40_000)
    outer = rng.uniform(2 * a, 3 * a, 30_000), rng.uniform(0, 2 * np.pi, 30_000)
    pts = []
    for r, phi in (inner, outer):
        p = np.stack([r * np.cos(phi), r * np.sin(phi)])
        pts += [p, -p]  # symmetric pairs: centroid at the origin
    ring = np.concatenate([np.tile([[a], [0.0]], 40_000), np.tile([[-a], [0.0]], 40_000),
                           np.tile([[0.0], [a]], 40_000), np.tile([[0.0], [-a]], 40_000)], axis=1)
    xy = np.concatenate(pts + [ring], axis=1)
    xy = xy[:, rng.permutation(xy.shape[1])]
    n = xy.shape[1]
    dt = torch.float32 if precision == 32 else torch.float64
    fxy = torch.from_numpy(np.ascontiguousarray(xy)).to("cuda", dt)
    status = torch.ones(n, dtype=torch.uint8, device="cuda")
    geom, _ = _trace(32, 100, seed=1, angles=(0.0,))
    ref = robast.psf(geom, status, fxy, precision=precision, windows=[(0, n)])[0]
    got = robast.psf_noalloc(status, fxy, [(0, n)], precision=precision)[0]
    _same(got, ref)
    # the crowded final bin is resolved by counting copies of each value: the exact
    # nearest-rank radius, identical to the allocating entry point's and from call to call
    assert got[3] == ref[3]
    assert robast.psf_noalloc(status, fxy, [(0, n)], precision=precision)[0][3] == got[3]
    x = xy.astype(np.float32 if precision == 32 else np.float64).astype(np.float64)
    r = np.sort(np.hypot(x[0] - ref[1], x[1] - ref[2]))
    assert got[3] == pytest.approx(r[int(math.ceil(0.8 * n)) - 1], rel=1e-12, abs=1e-15)
    assert abs(got[3] - a) < 1e-6
    geom.close()
