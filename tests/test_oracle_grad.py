"""Pins of the oracle's frozen-path gradients (forward-mode dual numbers).

Against closed forms (a flat mirror tilted by beta turns the reflected ray by
2 beta, so the spot moves by 2 L per radian; an asphere term A1 rho on a
paraboloid changes its focal length to f / (1 + 4 f A1)) and against central
finite differences (h = 1e-6) of the frozen-path objective itself.
Relative error: |g - g_ref| / max(|g_ref|, 1e-3 max|g_ref|).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _rel(g, ref):
    scale = max(np.max(np.abs(ref)), 1e-300)
    return np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * scale)


def test_flat_mirror_tilt_moves_centroid_by_twice_the_distance():
    L = 7.0
    mirror = W.Surface("sag", "mirror", "circle", ap=(1.0, 0, 0, 0))
    focal = W.Surface("sag", "focal", "rect", origin=(0, 0, L), rot=W.FACING_DOWN, ap=(2.0, 2.0, 0, 0))
    scene = W.Scene("flat", [mirror, focal], [W.Material([400.0], [1.0])], [W.Medium()], 10.0, L)
    rng = np.random.default_rng(0)
    m = 200
    o = np.stack([rng.uniform(-0.5, 0.5, m), rng.uniform(-0.5, 0.5, m), np.full(m, 3.0)])
    # shift the bundle so the focal plane's back does not shadow it: start below the focal plane
    b = W.Bundle(o, np.repeat([[0.0], [0.0], [-1.0]], m, axis=1), np.full(m, 400.0))
    _, gx = oracle.objective(scene, b, "centroid_x")
    _, gy = oracle.objective(scene, b, "centroid_y")
    # d(centroid x)/d(tilt about local y) = 2 L ; tilt about local x moves world y by -2 L, focal local y = -world y
    assert abs(gx[0, 1] - 2 * L) < 1e-9 * L
    assert abs(gy[0, 0] - 2 * L) < 1e-9 * L
    assert abs(gx[0, 0]) < 1e-9 and abs(gy[0, 1]) < 1e-9


def test_paraboloid_asphere_term_against_closed_form_msr():
    f = 10.0
    A0 = 2e-5
    mirror = W.Surface("sag", "mirror", "circle", curv=1 / (2 * f), conic=-1.0, asph=(A0,) + (0.0,) * 7,
                       ap=(2.0, 0, 0, 0))
    focal = W.Surface("sag", "focal", "rect", origin=(0, 0, f), rot=W.FACING_DOWN, ap=(0.5, 0.5, 0, 0))
    scene = W.Scene("parab", [mirror, focal], [W.Material([400.0], [1.0])], [W.Medium()], 20.0, f)
    rng = np.random.default_rng(1)
    m = 400
    r = 0.6 + 1.3 * np.sqrt(rng.random(m))
    ph = rng.uniform(0, 2 * np.pi, m)
    o = np.stack([r * np.cos(ph), r * np.sin(ph), np.full(m, 12.0)])
    b = W.Bundle(o, np.repeat([[0.0], [0.0], [-1.0]], m, axis=1), np.full(m, 400.0))
    val, g = oracle.objective(scene, b, "msr")

    def closed(A1):
        fp = f / (1 + 4 * f * A1)          # focal length of z = rho (1/4f + A1)
        zm = r * r / (4 * fp)
        s = (f - zm) / (fp - zm)           # reflected ray towards the focus (0, 0, fp), crossing z = f
        x = o[0] * (1 - s)
        y = -o[1] * (1 - s)                # focal frame faces down: local y = -world y
        return np.mean((x - x.mean()) ** 2 + (y - y.mean()) ** 2)

    assert val == pytest.approx(closed(A0), rel=1e-9)
    h = 1e-10
    ref = (closed(A0 + h) - closed(A0 - h)) / (2 * h)
    assert g[0, 2] == pytest.approx(ref, rel=1e-5)


def _fd(scene, b, objective, sid, k, h=1e-6, **kw):
    ns = len(scene.surfaces)
    dp = np.zeros((ns, oracle.N_PARAM))
    dm = np.zeros((ns, oracle.N_PARAM))
    dp[sid, k] = h
    dm[sid, k] = -h
    vp, _ = oracle.objective(scene, b, objective, delta=dp, grad=False, **kw)
    vm, _ = oracle.objective(scene, b, objective, delta=dm, grad=False, **kw)
    return (vp - vm) / (2 * h)


def test_duals_match_central_differences_on_the_dish():
    scene, b = W.lst_workload(600, seed=2, angles_deg=(1.0,))
    _, g = oracle.objective(scene, b, "msr", seed=3)
    counts = {}
    for sid, s in enumerate(scene.surfaces):
        if s.role == "mirror":
            counts[sid] = abs(g[sid]).sum()
    facets = sorted(counts, key=counts.get)[-3:]
    checks = []
    for sid in facets:
        for k in (0, 1, 2, 3, 9):
            checks.append((sid, k, g[sid, k], _fd(scene, b, "msr", sid, k, seed=3)))
    ref = np.array([c[3] for c in checks])
    got = np.array([c[2] for c in checks])
    assert np.max(_rel(got, ref)) < 1e-6, checks


def test_duals_match_central_differences_on_a_cone_soft_ce():
    scene = W.cone_scene(n_variants=1, seed=0)
    H = W.cone_heights(1)[0]
    bs = [W.hexagon_bundle(400, W.CONE_A_IN, H + W.CONE_WINDOW + 1e-4, math.radians(a), seed=3, stream=50 + i)
          for i, a in enumerate((10.0, 25.0, 33.0))]
    b = W.concat(bs)
    _, g = oracle.objective(scene, b, "soft_ce", seed=4, max_bounces=30)
    cone = 1
    got = g[cone, 10:16]
    # the sigmoid (tau = 0.5 mm) is steep in the control points: central differences converge as h^2
    # (measured 4.8e-4, 4.8e-6, 5e-8 relative at h = 1e-6, 1e-7, 1e-8 m), so the step is 1e-8 m here
    ref = np.array([_fd(scene, b, "soft_ce", cone, 10 + k, h=1e-8, seed=4, max_bounces=30) for k in range(6)])
    assert np.any(np.abs(ref) > 0)
    assert np.max(_rel(got, ref)) < 1e-6, (got, ref)


def _fd_h(scene, b, objective, sid, k, h, **kw):
    return _fd(scene, b, objective, sid, k, h=h, **kw)


def test_duals_cover_both_mirrors_of_a_two_mirror_system():
    """Schwarzschild-Couder-like optics: every detected photon reflects off a
    primary panel and then a secondary panel, so both carry gradients; the
    duals match central differences for tilts and aspheric terms of panels of
    each mirror (steps scaled so each moves the sag by ~1e-7 m at the rim)."""
    scene, b = W.sct_workload(150, seed=1, angles_deg=(0.0, 1.5))
    _, g = oracle.objective(scene, b, "msr", seed=2)
    prim = [i for i, s in enumerate(scene.surfaces) if s.role == "mirror" and s.origin[2] == 0.0]
    sec = [i for i, s in enumerate(scene.surfaces) if s.role == "mirror" and s.origin[2] != 0.0]
    assert prim and sec
    # the panels of each mirror with the largest gradient
    pick = [max(prim, key=lambda i: abs(g[i]).sum()), max(sec, key=lambda i: abs(g[i]).sum())]
    assert all(abs(g[i, :2]).sum() > 0 for i in pick)
    checks = []
    for sid in pick:
        rmax = scene.surfaces[sid].ap[1]
        for k, h in ((0, 1e-6), (1, 1e-6), (2, 1e-7 / rmax ** 2), (3, 1e-7 / rmax ** 4)):
            checks.append((sid, k, g[sid, k], _fd_h(scene, b, "msr", sid, k, h, seed=2)))
    got = np.array([c[2] for c in checks])
    ref = np.array([c[3] for c in checks])
    assert np.max(_rel(got, ref)) < 1e-5, checks


def test_duals_cover_paths_through_more_mirrors_than_one_replay_tracks():
    """A zigzag of six distinct flat mirrors (three on the floor, three on the
    ceiling) ends on a vertical focal plane: every photon meets all six, more
    than one dual replay carries, so the replay runs in groups; each mirror's
    tilt gradient matches central differences."""
    surfs = []
    for k in range(6):
        up = k % 2 == 1
        surfs.append(W.Surface("sag", "mirror", "circle", origin=(float(k), 0.0, 1.0 if up else 0.0),
                               rot=W.FACING_DOWN if up else (1, 0, 0, 0, 1, 0, 0, 0, 1), ap=(0.45, 0, 0, 0)))
    surfs.append(W.Surface("sag", "focal", "rect", origin=(5.5, 0.0, 0.5), rot=W.frame_from_axis((-1.0, 0.0, 0.0)),
                           ap=(1.0, 1.0, 0, 0)))
    scene = W.Scene("zigzag", surfs, [W.Material([400.0], [1.0])], [W.Medium()], 10.0, 1.0)
    rng = np.random.default_rng(7)
    m = 40
    o = np.stack([np.full(m, -0.5), rng.uniform(-0.05, 0.05, m), 0.5 + rng.uniform(-0.02, 0.02, m)])
    d = np.repeat([[1.0], [0.0], [-1.0]], m, axis=1) / math.sqrt(2.0)
    b = W.Bundle(o, d, np.full(m, 400.0))
    r = oracle.trace(scene, b, seed=0)
    assert np.all(r["status"] == W.DETECTED) and np.all(r["bounces"] == 7)
    _, g = oracle.objective(scene, b, "msr", seed=0)
    got = np.array([g[sid, 1] for sid in range(6)])
    ref = np.array([_fd(scene, b, "msr", sid, 1, seed=0) for sid in range(6)])
    assert np.all(np.abs(got) > 0)  # a tilt about local y moves every spot
    assert np.max(_rel(got, ref)) < 1e-6, (got, ref)
    # tilts about local x move the spots across the plane of incidence symmetrically: no MSR change
    assert np.max(np.abs(g[:6, 0])) < 1e-12 * np.max(np.abs(got))
