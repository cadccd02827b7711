"""Photon-track records of the oracle, checked against geometry and against
the oracle's own per-photon results (CPU).

On the single spherical mirror (R = 10 m, vertex at the origin, concave to
+z) every recorded mirror point lies on the sphere |p - (0, 0, R)| = R, every
focal point on the plane z = 5 m inside the 0.3 m square, and each photon's
records are one per bounce, ending at the trace's final point, last surface
and status.
"""
import numpy as np

import oracle
import workloads as W

MIRROR, FOCAL = 0, 1


def test_track_records_lie_on_the_surfaces_and_end_at_the_trace_result():
    scene, b = W.sphere_workload(2_000, seed=3)
    ref = oracle.trace(scene, b, seed=7)
    first, count = 100, 700
    pts, info = oracle.track(scene, b, first, count, seed=7)
    assert len(pts) > 0
    assert np.all((info[:, 0] >= first) & (info[:, 0] < first + count))
    R = 10.0
    on_mirror = info[:, 2] == MIRROR
    assert on_mirror.any()
    r = np.linalg.norm(pts[on_mirror] - np.array([0.0, 0.0, R]), axis=1)
    assert np.max(np.abs(r - R)) < 1e-9
    on_focal = info[:, 2] == FOCAL
    assert on_focal.any()
    assert np.max(np.abs(pts[on_focal, 2] - 5.0)) < 1e-9
    assert np.all(np.abs(pts[on_focal, :2]) <= 0.15 + 1e-12)
    for i in range(first, first + count):
        rec = info[:, 0] == i
        k = int(rec.sum())
        assert k == int(ref["bounces"][i]), i
        if k == 0:
            assert ref["status"][i] == W.ESCAPED
            continue
        order = np.argsort(info[rec, 1])
        bi, st, sid = info[rec, 1][order], info[rec, 3][order], info[rec, 2][order]
        assert np.array_equal(bi, np.arange(k))          # one record per bounce, 0-based
        if ref["status"][i] == W.ESCAPED:  # an escape is not an interaction: no record ends the path
            assert np.all(st == 0)
        else:
            assert np.all(st[:-1] == 0) and st[-1] == ref["status"][i]  # only the last one terminates
        assert sid[-1] == ref["last_surface"][i]
        assert np.allclose(pts[rec][order][-1], ref["hit"][:, i], rtol=0, atol=1e-12)
