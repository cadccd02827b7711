"""Closed-form pins of oracle functions that the trace tests reach only indirectly.

* Even-asphere terms A1..A8 (Sec. 2.2, aspheric disk): a ray parallel to the
  axis at height h meets a pure-polynomial sag (c = 0) at z = sum_i A_i h^(2i),
  and the surface slope there is dz/dh = sum_i 2 i A_i h^(2i-1).  Each term is
  checked alone and all eight together, through the hit point, the front
  normal and the reflected direction of a traced photon.
* The box obscuration (camera box, Sec. 3): entry distance and outward normal
  for rays aimed at each face from outside, the far face from inside, edges
  and corners, and misses.
* The spot-diagram reduction (Fig. 1 g-i reading): centroid and nearest-rank
  R80 of hand-built point sets whose answer is known by construction.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import metrics
from workloads import DETECTED, ESCAPED, OBSCURED


def _bundle(origins, dirs, lam=400.0):
    o = np.ascontiguousarray(np.asarray(origins, np.float64).T)
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return W.Bundle(o, np.ascontiguousarray(d.T), np.full(o.shape[1], float(lam)))


# ------------------------------------------------------------ asphere terms
H_MAX = 1.0


def _poly_mirror(coeffs):
    return W.Surface("sag", "mirror", "circle", curv=0.0, asph=tuple(coeffs), ap=(1.2 * H_MAX, 0, 0, 0))


def _sag_closed(coeffs, h):
    return sum(a * h ** (2 * i) for i, a in enumerate(coeffs, start=1))


def _dsag_dh_closed(coeffs, h):
    return sum(2 * i * a * h ** (2 * i - 1) for i, a in enumerate(coeffs, start=1))


COEFF_CASES = []
for _i in range(8):
    _c = [0.0] * 8
    # each term alone gives a sag of +-0.04 m at the rim: well inside Newton's basin
    _c[_i] = (0.04 if _i % 2 == 0 else -0.04) / H_MAX ** (2 * (_i + 1))
    COEFF_CASES.append((f"A{_i + 1}", _c))
COEFF_CASES.append(("A1..A8", [0.02, -0.013, 0.011, -0.007, 0.005, -0.004, 0.003, -0.002]))


@pytest.mark.parametrize("name,coeffs", COEFF_CASES, ids=[c[0] for c in COEFF_CASES])
def test_asphere_terms_hit_height_and_normal_closed_form(name, coeffs):
    mirror = _poly_mirror(coeffs)
    z0 = 2.0
    for h in (0.13, 0.37, 0.61, 0.83, 0.97):
        for phi in (0.0, 0.7, 2.9):
            x, y = h * math.cos(phi), h * math.sin(phi)
            res = oracle.intersect(mirror, [x, y, z0], [0.0, 0.0, -1.0])
            assert res is not None, (name, h)
            t, n, lp = res
            z_exp = _sag_closed(coeffs, h)
            assert abs((z0 - t) - z_exp) < 1e-12, (name, h, z0 - t, z_exp)
            assert abs(lp[2] - z_exp) < 1e-12
            s = _dsag_dh_closed(coeffs, h)
            # the surface z = g(h) has the upward normal (-g'(h) cos phi, -g'(h) sin phi, 1) / norm
            ne = np.array([-s * math.cos(phi), -s * math.sin(phi), 1.0])
            ne /= np.linalg.norm(ne)
            assert np.max(np.abs(n - ne)) < 1e-12, (name, h, n, ne)


@pytest.mark.parametrize("name,coeffs", COEFF_CASES, ids=[c[0] for c in COEFF_CASES])
def test_asphere_terms_reflect_by_twice_the_slope_angle(name, coeffs):
    """A photon going down the axis direction reflects off the polynomial mirror
    (reflectivity 1) at the closed-form height and leaves at twice the surface
    slope angle atan(dz/dh) from the axis, in the meridional plane."""
    scene = W.Scene("poly", [_poly_mirror(coeffs)], [W.Material([400.0], [1.0])], [W.Medium()], 4.0, 1.0)
    hs = np.array([0.21, 0.44, 0.58, 0.76, 0.9])
    phis = np.array([0.3, 1.9, 3.3, 4.4, 5.8])
    origins = [[h * math.cos(p), h * math.sin(p), 1.5] for h, p in zip(hs, phis)]
    r = oracle.trace(scene, _bundle(origins, [[0, 0, -1]] * len(hs)), n_threads=1)
    assert np.all(r["status"] == ESCAPED) and np.all(r["bounces"] == 1)
    for k, (h, p) in enumerate(zip(hs, phis)):
        assert abs(r["hit"][2, k] - _sag_closed(coeffs, h)) < 1e-12
        alpha = math.atan(_dsag_dh_closed(coeffs, h))
        d = r["dir"][:, k]
        radial = d[0] * math.cos(p) + d[1] * math.sin(p)
        tang = -d[0] * math.sin(p) + d[1] * math.cos(p)
        # incoming (0, 0, -1) mirrored about a normal tilted by alpha towards -radial:
        # outgoing = (-sin 2 alpha radial, cos 2 alpha up)
        assert abs(tang) < 1e-13
        assert abs(radial + math.sin(2 * alpha)) < 1e-12, (name, h)
        assert abs(d[2] - math.cos(2 * alpha)) < 1e-12, (name, h)


# ------------------------------------------------------------------- box
HX, HY, HZ = 1.5, 0.75, 1.0


def _box(origin=(0.0, 0.0, 0.0), rot=(1, 0, 0, 0, 1, 0, 0, 0, 1)):
    return W.Surface("box", "obscuration", origin=origin, rot=rot, prm=(HX, HY, HZ, 0, 0, 0, 0, 0))


FACES = [  # (axis, sign, half extent)
    (0, +1, HX), (0, -1, HX), (1, +1, HY), (1, -1, HY), (2, +1, HZ), (2, -1, HZ)]


@pytest.mark.parametrize("axis,sign,hw", FACES)
def test_box_entry_face_distance_and_outward_normal(axis, sign, hw):
    """A ray from outside aimed (obliquely) at the middle region of one face
    enters through that face: t = (distance along the axis) / |d_axis|, the
    normal is that face's outward normal."""
    box = _box()
    rng = np.random.default_rng(10 * axis + (sign > 0))
    ext = np.array([HX, HY, HZ])
    for _ in range(20):
        target = rng.uniform(-0.8, 0.8, 3) * ext
        target[axis] = sign * hw
        d = rng.normal(0, 0.2, 3)
        d[axis] = -sign * 1.0
        d /= np.linalg.norm(d)
        start_dist = rng.uniform(0.5, 5.0)
        p = target - start_dist * d
        res = oracle.intersect(box, p, d)
        assert res is not None
        t, n, lp = res
        assert abs(t - start_dist) < 1e-12
        ne = np.zeros(3)
        ne[axis] = sign
        assert np.array_equal(n, ne)
        assert np.max(np.abs(lp - target)) < 1e-12


@pytest.mark.parametrize("axis,sign,hw", FACES)
def test_box_from_inside_hits_the_far_face(axis, sign, hw):
    box = _box()
    rng = np.random.default_rng(100 + 10 * axis + (sign > 0))
    ext = np.array([HX, HY, HZ])
    for _ in range(20):
        p = rng.uniform(-0.5, 0.5, 3) * ext
        d = rng.normal(0, 0.05, 3)
        d[axis] = sign * 1.0
        d /= np.linalg.norm(d)
        t, n, lp = oracle.intersect(box, p, d)
        assert abs(t - (hw - sign * p[axis]) / abs(d[axis])) < 1e-12
        ne = np.zeros(3)
        ne[axis] = sign
        assert np.array_equal(n, ne)
        assert abs(lp[axis] - sign * hw) < 1e-12


def test_box_edges_corners_and_misses():
    box = _box()
    # corner: the ray along the body diagonal from outside reaches (HX, HY, HZ)
    corner = np.array([HX, HY, HZ])
    d = -corner / np.linalg.norm(corner)
    p = corner - 3.0 * d
    t, n, lp = oracle.intersect(box, p, d)
    assert abs(t - 3.0) < 1e-12 and np.max(np.abs(lp - corner)) < 1e-12
    # the normal is the outward normal of one of the three faces meeting there
    assert any(np.array_equal(n, e) for e in np.eye(3))
    # edge x = HX, y = -HY at z = 0.3: approached in the x-y plane at 45 degrees
    edge = np.array([HX, -HY, 0.3])
    d = np.array([-1.0, 1.0, 0.0]) / math.sqrt(2.0)
    t, n, lp = oracle.intersect(box, edge - 2.0 * d, d)
    assert abs(t - 2.0) < 1e-12 and np.max(np.abs(lp - edge)) < 1e-12
    assert np.array_equal(n, [1.0, 0.0, 0.0]) or np.array_equal(n, [0.0, -1.0, 0.0])
    # a ray passing just outside a face misses; one pointing away misses
    assert oracle.intersect(box, [HX + 1e-6, -5.0, 0.0], [0.0, 1.0, 0.0]) is None
    assert oracle.intersect(box, [0.0, 0.0, HZ + 1.0], [0.0, 0.0, 1.0]) is None
    # a ray parallel to a slab, outside it, misses even when aimed at the box's x-y footprint
    assert oracle.intersect(box, [-5.0, 0.0, HZ + 0.01], [1.0, 0.0, 0.0]) is None
    # the same ray inside the slab enters through the x = -HX face
    t, n, lp = oracle.intersect(box, [-5.0, 0.2, HZ - 0.01], [1.0, 0.0, 0.0])
    assert abs(t - (5.0 - HX)) < 1e-12 and np.array_equal(n, [-1.0, 0.0, 0.0])


def test_box_in_a_rotated_offset_frame_and_in_a_trace():
    """World geometry of a rotated, shifted box: the hit lies on the rotated
    face, the world normal is the rotated face normal; traced, the photon is
    OBSCURED at that point after one bounce."""
    ang = 0.4
    rot = (math.cos(ang), math.sin(ang), 0.0, -math.sin(ang), math.cos(ang), 0.0, 0.0, 0.0, 1.0)
    o = np.array([2.0, -1.0, 3.0])
    box = _box(tuple(o), rot)
    ex = np.array(rot[0:3])  # local x axis in world coordinates
    target = o + HX * ex + 0.2 * np.array(rot[3:6]) - 0.3 * np.array([0, 0, 1.0])
    d = -ex
    p = target + 4.0 * ex
    t, n, lp = oracle.intersect(box, p, d)
    assert abs(t - 4.0) < 1e-12
    assert np.max(np.abs(n - ex)) < 1e-15
    assert np.max(np.abs(lp - np.array([HX, 0.2, -0.3]))) < 1e-12
    scene = W.Scene("box", [box], [W.Material([400.0], [1.0])], [W.Medium()], 10.0, 1.0)
    r = oracle.trace(scene, _bundle([p], [d]), n_threads=1)
    assert r["status"][0] == OBSCURED and r["bounces"][0] == 1
    assert np.max(np.abs(r["hit"][:, 0] - target)) < 1e-12


# -------------------------------------------------------------- spot metrics
def test_psf_centroid_and_nearest_rank_r80_by_construction():
    """Seven detected points around c = (0.3, -0.2): c itself and the pairs
    c +- v_k with |v_k| = 1, 2, 3 mm.  The centroid is c; the sorted radii are
    0, 1, 1, 2, 2, 3, 3 mm and the nearest rank ceil(0.8 * 7) = 6 picks the
    sixth, 3 mm.  Undetected photons far away must not count."""
    c = np.array([0.3, -0.2])
    pts = [c]
    for k, ang in zip((1, 2, 3), (0.3, 2.0, 4.1)):
        v = 1e-3 * k * np.array([math.cos(ang), math.sin(ang)])
        pts += [c + v, c - v]
    xy = np.array(pts).T
    junk = np.array([[50.0, -40.0, 7.0], [9.0, 3.0, -60.0]])
    xy_all = np.concatenate([xy, junk], axis=1)
    st = np.array([DETECTED] * 7 + [OBSCURED, 2, ESCAPED], np.uint8)
    m = metrics.psf(st, xy_all)
    assert m["n_detected"] == 7
    assert abs(m["cx"] - 0.3) < 1e-15 and abs(m["cy"] + 0.2) < 1e-15
    assert abs(m["r80"] - 3e-3) < 1e-15


def test_psf_nearest_rank_index_for_several_counts():
    """Points on rings of radii 1..N (one point each, arranged in opposite pairs
    so the centroid is the origin, plus the origin itself for odd N): R80 is
    the radius of sorted index ceil(0.8 N) - 1."""
    for n_pairs in (1, 2, 3, 5, 8, 13):
        for with_centre in (False, True):
            pts = [[0.0, 0.0]] if with_centre else []
            radii = [0.0] if with_centre else []
            for k in range(1, n_pairs + 1):
                a = 0.7 * k
                pts += [[k * math.cos(a), k * math.sin(a)], [-k * math.cos(a), -k * math.sin(a)]]
                radii += [k, k]
            xy = np.array(pts).T
            n = xy.shape[1]
            m = metrics.psf(np.full(n, DETECTED, np.uint8), xy)
            expect = sorted(radii)[math.ceil(0.8 * n) - 1]
            assert abs(m["cx"]) < 1e-12 and abs(m["cy"]) < 1e-12
            assert abs(m["r80"] - expect) < 1e-12, (n, m["r80"], expect)
    # nothing detected: NaN statistics
    m = metrics.psf(np.full(4, OBSCURED, np.uint8), np.zeros((2, 4)))
    assert m["n_detected"] == 0 and math.isnan(m["r80"])


def test_effective_area_and_collection_efficiency():
    st = np.array([DETECTED, OBSCURED, DETECTED, ESCAPED], np.uint8)
    assert metrics.collection_efficiency(st) == 0.5
    assert abs(metrics.effective_area(st, 2.0) - 0.5 * math.pi * 4.0) < 1e-15
