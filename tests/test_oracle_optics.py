"""Pins of the FP64 oracle against closed forms, invariants and textbook optics.

None of these re-type the oracle's own formulas: each checks a traced result
against an independent geometric derivation (mirror equation, spherical
aberration of a sphere, the focusing property of a paraboloid, the
Davies-Cotton facet alignment, the edge-ray theorem of the 2D compound
parabolic concentrator, energy conservation through Fresnel transmission
amplitudes, the parallel-slab invariant, the doubling of a mirror tilt).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import DETECTED, ABSORBED, OBSCURED, ESCAPED, MAX_BOUNCES, ERROR


def _trace(scene, bundle, **kw):
    return oracle.trace(scene, bundle, n_threads=4, **kw)


def _bundle(origins, dirs, lam=400.0):
    o = np.ascontiguousarray(np.asarray(origins, np.float64).T)
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return W.Bundle(o, np.ascontiguousarray(d.T), np.full(o.shape[1], float(lam)))


# ------------------------------------------------------------ single sphere
def test_sphere_spherical_aberration_closed_form():
    """Sec. 3 workload 1.  A ray parallel to the axis at height h meets the
    sphere (centre on axis at R) at z_m = R - sqrt(R^2 - h^2); the normal there
    makes alpha with the axis, sin(alpha) = h/R; the reflected ray makes
    2 alpha and crosses z = f at radius h - (f - z_m) tan(2 alpha)."""
    scene, b = W.sphere_workload(20000, seed=3)
    r = _trace(scene, b)
    R, f = 10.0, 5.0
    x0, y0 = b.origins[0], b.origins[1]
    h = np.hypot(x0, y0)
    det = r["status"] == DETECTED
    assert det.sum() > 10000
    hd = h[det]
    zm = R - np.sqrt(R * R - hd * hd)
    alpha = np.arcsin(hd / R)
    rad = hd - (f - zm) * np.tan(2 * alpha)
    ex = x0[det] * rad / hd
    ey = y0[det] * rad / hd
    fx, fy = r["focal_xy"][0][det], -r["focal_xy"][1][det]  # focal frame faces -z: local y = -world y
    assert np.max(np.abs(fx - ex)) < 1e-12 * f
    assert np.max(np.abs(fy - ey)) < 1e-12 * f
    # world hit point is on the focal plane
    assert np.max(np.abs(r["hit"][2][det] - f)) < 1e-12 * f


def test_sphere_status_map():
    scene, b = W.sphere_workload(20000, seed=4)
    r = _trace(scene, b)
    x0, y0 = b.origins[0], b.origins[1]
    h = np.hypot(x0, y0)
    shadow = (np.abs(x0) <= 0.15) & (np.abs(y0) <= 0.15)
    st = r["status"]
    assert np.all(st[shadow] == OBSCURED)                      # back of the focal plane
    assert np.all(st[~shadow & (h > 0.5)] == ESCAPED)          # outside the mirror
    on = ~shadow & (h <= 0.5)
    assert np.all(np.isin(st[on], [DETECTED, ABSORBED]))
    assert np.all(r["bounces"][shadow] == 1)
    assert np.all(r["bounces"][~shadow & (h > 0.5)] == 0)
    assert np.all(r["bounces"][on & (st == DETECTED)] == 2)
    # survival is binomial with p = 0.9
    n = on.sum()
    k = (st[on] == DETECTED).sum()
    assert abs(k / n - 0.9) < 5 * math.sqrt(0.09 / n)


# ---------------------------------------------------------- paraboloid focus
def test_paraboloid_focuses_on_axis_rays_exactly():
    f = 28.0
    mirror = W.Surface("sag", "mirror", "circle", curv=1.0 / (2 * f), conic=-1.0, ap=(12.0, 0, 0, 0))
    focal = W.Surface("sag", "focal", "rect", origin=(0, 0, f), rot=W.FACING_DOWN, ap=(0.05, 0.05, 0, 0))
    mat = W.Material(lam=[400.0], refl=[1.0])
    scene = W.Scene("parab", [mirror, focal], [mat], [W.Medium()], 46.6, f)
    b = W.disk_bundle(20000, 11.9, 32.0, 0.0, (400.0, 400.0), seed=5)
    r = _trace(scene, b)
    det = r["status"] == DETECTED
    shadow = (np.abs(b.origins[0]) <= 0.05) & (np.abs(b.origins[1]) <= 0.05)
    assert det.sum() == (~shadow).sum()
    assert np.max(np.hypot(*r["focal_xy"][:, det])) < 1e-12 * f


def test_asphere_newton_matches_closed_form_paraboloid():
    """The paraboloid z = rho / 4f written as a pure polynomial sag (c = 0,
    A1 = 1/4f) goes through the Newton path; its hits must coincide with the
    closed-form quadric path (c = 1/2f, k = -1)."""
    f = 7.0
    quad = W.Surface("sag", "mirror", "circle", curv=1.0 / (2 * f), conic=-1.0, ap=(3.0, 0, 0, 0))
    poly = W.Surface("sag", "mirror", "circle", curv=0.0, asph=(1.0 / (4 * f),) + (0.0,) * 7, ap=(3.0, 0, 0, 0))
    rng = np.random.default_rng(0)
    for _ in range(200):
        p = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), 10.0])
        d = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), -1.0])
        d /= np.linalg.norm(d)
        a = oracle.intersect(quad, p, d)
        b = oracle.intersect(poly, p, d)
        assert (a is None) == (b is None)
        if a is not None:
            assert abs(a[0] - b[0]) < 1e-11
            assert np.max(np.abs(a[1] - b[1])) < 1e-11


# ----------------------------------------------------------- Davies-Cotton
def test_davies_cotton_facet_centres_image_on_axis():
    """Facets centred on a sphere of radius f around the focus, each a sphere
    of radius 2f aimed at (0, 0, 2f): the on-axis ray through each facet centre
    is reflected exactly through the focus."""
    f = 10.0
    surfs = [W.Surface("sag", "focal", "circle", origin=(0, 0, f), rot=W.FACING_DOWN, ap=(0.01, 0, 0, 0))]
    centres = []
    for k in range(7):
        rho = 0.0 if k == 0 else 1.2
        phi = 2 * math.pi * k / 6
        x, y = rho * math.cos(phi), rho * math.sin(phi)
        z = f - math.sqrt(f * f - x * x - y * y)
        c = np.array([x, y, z])
        n = np.array([0, 0, 2 * f]) - c
        surfs.append(W.Surface("sag", "mirror", "hexagon", origin=tuple(c), rot=W.frame_from_axis(n),
                               curv=1.0 / (2 * f), ap=(0.5, 0, 0, 0)))
        centres.append(c)
    scene = W.Scene("dc", surfs, [W.Material([400.0], [1.0])], [W.Medium()], 20.0, f)
    # start each ray just above its facet centre (below the focal disk)
    o = [c + np.array([0, 0, 1.0]) for c in centres[1:]]
    r = _trace(scene, _bundle(o, [[0, 0, -1]] * len(o)))
    assert np.all(r["status"] == DETECTED)
    assert np.max(np.hypot(*r["focal_xy"])) < 1e-12 * f


def test_davies_cotton_spot_against_sphere_centre_formula():
    """Random rays on one Davies-Cotton facet: the traced focal point equals an
    independent ray-sphere construction (sphere written by its centre)."""
    f = 10.0
    x, y = 1.2, 0.0
    c = np.array([x, y, f - math.sqrt(f * f - x * x)])
    n = np.array([0, 0, 2 * f]) - c
    n /= np.linalg.norm(n)
    C = c + 2 * f * n  # centre of the facet sphere
    focal = W.Surface("sag", "focal", "rect", origin=(0, 0, f), rot=W.FACING_DOWN, ap=(1.0, 1.0, 0, 0))
    facet = W.Surface("sag", "mirror", "hexagon", origin=tuple(c), rot=W.frame_from_axis(n), curv=1.0 / (2 * f),
                      ap=(0.5, 0, 0, 0))
    scene = W.Scene("dc1", [facet, focal], [W.Material([400.0], [1.0])], [W.Medium()], 20.0, f)
    rng = np.random.default_rng(1)
    m = 500
    o = np.stack([x + rng.uniform(-0.4, 0.4, m), y + rng.uniform(-0.4, 0.4, m), np.full(m, 5.0)], 1)
    o = o[(np.abs(o[:, 0] - x) > 0.0) & ~((np.abs(o[:, 0]) <= 1.0) & (np.abs(o[:, 1]) <= 1.0))]
    r = _trace(scene, _bundle(o, [[0, 0, -1]] * len(o)))
    det = r["status"] == DETECTED
    assert det.sum() > 0
    for i in np.where(det)[0]:
        p = o[i]
        d = np.array([0.0, 0.0, -1.0])
        # |p + t d - C| = 2f; the ray starts inside the facet sphere, so the
        # concave side is met at the larger root
        oc = p - C
        bq = np.dot(oc, d)
        t = -bq + math.sqrt(bq * bq - (np.dot(oc, oc) - 4 * f * f))
        q = p + t * d
        nn = (C - q) / (2 * f)
        rr = d - 2 * np.dot(d, nn) * nn
        s = (f - q[2]) / rr[2]
        e = q + s * rr
        assert abs(r["focal_xy"][0][i] - e[0]) < 1e-11 and abs(-r["focal_xy"][1][i] - e[1]) < 1e-11


# ---------------------------------------------------------- 2D Winston cone
def _winston_2d_scene():
    P0, P1, P2 = W.winston_profile()
    surfs = [W.Surface("sag", "focal", "hexagon", ap=(W.CONE_A_OUT, 0, 0, 0)),
             W.Surface("hexcone", "mirror", material=0, prm=(P0[0], P0[1], P1[0], P1[1], P2[0], P2[1], 0, 0))]
    return W.Scene("winston2d", surfs, [W.Material([400.0], [1.0])], [W.Medium()], 0.1, 0.05), P2[1]


@pytest.mark.parametrize("theta_deg,expected", [(0.0, 1.0), (10.0, 1.0), (20.0, 1.0), (29.0, 1.0), (29.9, 1.0),
                                                (30.1, 0.0), (31.0, 0.0), (35.0, 0.0), (45.0, 0.0)])
def test_ideal_2d_winston_cutoff(theta_deg, expected):
    """Rays confined to the y = 0 plane meet only the two flats facing +-x, so
    the hexagonal Winston cone is exactly the 2D compound parabolic
    concentrator with acceptance 30 deg: transmission 1 below, 0 above."""
    scene, H = _winston_2d_scene()
    m = 4000
    x = np.linspace(-W.CONE_A_IN * 0.999, W.CONE_A_IN * 0.999, m)
    th = math.radians(theta_deg)
    o = np.stack([x, np.zeros(m), np.full(m, H + 1e-9)], 1)
    r = _trace(scene, _bundle(o, [[math.sin(th), 0.0, -math.cos(th)]] * m), max_bounces=50)
    ce = (r["status"] == DETECTED).mean()
    assert ce == expected, (theta_deg, ce, np.bincount(r["status"]))


def test_winston_bezier_points_lie_on_the_parabola():
    """Every reflection point on the Winston wall satisfies the parabola's
    focus-directrix definition: distance to the focus (-a', 0) equals the
    distance to the directrix (in the wall's (q, z) half-plane)."""
    scene, H = _winston_2d_scene()
    th = math.radians(30.0)
    a = W.CONE_A_OUT
    fp = a * (1 + math.sin(th))
    F = np.array([-a, 0.0])
    up = np.array([-math.sin(th), math.cos(th)])
    V = F - fp * up
    wall = scene.surfaces[1]
    rng = np.random.default_rng(2)
    for _ in range(300):
        xq = rng.uniform(-0.02, 0.02)
        ang = math.radians(rng.uniform(5, 40))
        p = np.array([xq, 0.0, H])
        d = np.array([math.sin(ang), 0.0, -math.cos(ang)])
        hit = oracle.intersect(wall, p, d)
        if hit is None:
            continue
        q = hit[2]
        qr = np.array([q[0], q[2]])  # wall facing +x: (q, z) = (x, z)
        if q[0] < 0:
            continue
        dist_f = np.linalg.norm(qr - F)
        dist_dir = np.dot(qr - V, up) + fp  # directrix at distance fp behind the vertex
        assert abs(dist_f - dist_dir) < 1e-12


# -------------------------------------------------------------- refraction
@pytest.mark.parametrize("n1,n2", [(1.0, 1.49), (1.49, 1.0), (1.0, 2.4), (1.33, 1.52)])
def test_fresnel_energy_conservation_via_transmission_amplitudes(n1, n2):
    for th in np.linspace(0.0, math.pi / 2 - 1e-3, 60):
        ci = math.cos(th)
        s2 = (n1 / n2) ** 2 * (1 - ci * ci)
        R = oracle.fresnel(n1, n2, ci)
        if s2 >= 1.0:
            assert R == 1.0
            continue
        ct = math.sqrt(1 - s2)
        ts = 2 * n1 * ci / (n1 * ci + n2 * ct)
        tp = 2 * n1 * ci / (n2 * ci + n1 * ct)
        T = (n2 * ct) / (n1 * ci) * 0.5 * (ts * ts + tp * tp)
        assert abs(R + T - 1.0) < 1e-13


def test_fresnel_normal_incidence_brewster_and_reciprocity():
    n1, n2 = 1.0, 1.5
    assert abs(oracle.fresnel(n1, n2, 1.0) - ((n1 - n2) / (n1 + n2)) ** 2) < 1e-15
    # at Brewster's angle the p-reflectance vanishes: R = Rs / 2, Rs = cos^2(2 thB)
    tb = math.atan(n2 / n1)
    assert abs(oracle.fresnel(n1, n2, math.cos(tb)) - 0.5 * math.cos(2 * tb) ** 2) < 1e-14
    # reciprocity: R(n1 -> n2, theta_i) = R(n2 -> n1, theta_t)
    for th in np.linspace(0.0, 1.4, 15):
        st = n1 / n2 * math.sin(th)
        assert abs(oracle.fresnel(n1, n2, math.cos(th)) - oracle.fresnel(n2, n1, math.sqrt(1 - st * st))) < 1e-13
    # TIR beyond the critical angle
    assert oracle.fresnel(1.5, 1.0, math.cos(math.asin(1 / 1.5) + 1e-6)) == 1.0


def test_pmma_index_textbook_value():
    # PMMA n_D (589.3 nm) is 1.4905 +- 0.001 in handbooks
    assert abs(oracle.refractive_index(W.PMMA, 589.3) - 1.4905) < 1e-3
    # normal dispersion
    assert oracle.refractive_index(W.PMMA, 350.0) > oracle.refractive_index(W.PMMA, 600.0)


def _slab_scene(thick=0.01, n_med=1.5, aperture=1.0):
    top = W.Surface("sag", "refract", "circle", origin=(0, 0, thick), medium_front=0, medium_back=1,
                    ap=(aperture, 0, 0, 0))
    bot = W.Surface("sag", "refract", "circle", origin=(0, 0, 0), medium_front=1, medium_back=0,
                    ap=(aperture, 0, 0, 0))
    return W.Scene("slab", [top, bot], [W.Material([400.0], [1.0])], [W.Medium(1.0), W.Medium(n_med)], 1.0, 1.0)


def test_parallel_slab_restores_direction_and_shifts_by_textbook_amount():
    """Snell at both faces of a parallel slab: the exit direction equals the
    entry direction and the lateral shift is T sin(ti - tt) / cos(tt)."""
    thick, nm = 0.01, 1.5
    scene = _slab_scene(thick, nm)
    m = 20000
    th = math.radians(35.0)
    o = np.tile([0.0, 0.0, 0.05], (m, 1))
    d = [[math.sin(th), 0.0, -math.cos(th)]] * m
    r = _trace(scene, _bundle(o, d))
    esc = r["status"] == ESCAPED
    down = esc & (r["dir"][2] < 0)
    assert down.sum() > 0.8 * m
    d_out = r["dir"][:, down]
    assert np.max(np.abs(d_out[0] - math.sin(th))) < 1e-14
    assert np.max(np.abs(d_out[2] + math.cos(th))) < 1e-14
    # exactly two refractions: hit point on the bottom face at the textbook position
    two = down & (r["bounces"] == 2)
    tt = math.asin(math.sin(th) / nm)
    x_entry = 0.05 - thick
    x_entry = (0.05 - thick) * math.tan(th)
    x_exit = x_entry + thick * math.tan(tt)
    assert np.max(np.abs(r["hit"][0][two] - x_exit)) < 1e-14
    # statistics of the first-face reflection against Fresnel R within 4 sigma
    R = oracle.fresnel(1.0, nm, math.cos(th))
    up1 = esc & (r["dir"][2] > 0) & (r["bounces"] == 1)
    k = up1.sum()
    assert abs(k / m - R) < 4 * math.sqrt(R * (1 - R) / m)


# --------------------------------------------------------- mirror details
def test_mirror_tilt_doubles_on_reflection():
    """A flat mirror tilted by alpha about its local x axis turns the reflected
    ray by 2 alpha."""
    for alpha in (1e-4, -3e-3, 0.05):
        m = W.Surface("sag", "mirror", "circle", tilt=(alpha, 0.0), ap=(1.0, 0, 0, 0))
        scene = W.Scene("tilt", [m], [W.Material([400.0], [1.0])], [W.Medium()], 1.0, 1.0)
        r = _trace(scene, _bundle([[0.0, 0.0, 1.0]], [[0, 0, -1]]))
        d = r["dir"][:, 0]
        ang = math.atan2(-d[1], d[2])  # rotation about +x of the +z direction
        assert abs(abs(ang) - 2 * abs(alpha)) < 1e-14
        # and the tilt about y moves x instead
        m2 = W.Surface("sag", "mirror", "circle", tilt=(0.0, alpha), ap=(1.0, 0, 0, 0))
        scene2 = W.Scene("tilt", [m2], [W.Material([400.0], [1.0])], [W.Medium()], 1.0, 1.0)
        d2 = _trace(scene2, _bundle([[0.0, 0.0, 1.0]], [[0, 0, -1]]))["dir"][:, 0]
        assert abs(d2[1]) < 1e-15 and abs(abs(math.atan2(d2[0], d2[2])) - 2 * abs(alpha)) < 1e-14


def test_roughness_spreads_reflection_by_twice_sigma():
    """Tilting the normal by a small angle delta turns the reflected ray by
    2 delta: per tangent axis the reflected direction spreads with 2 sigma."""
    sigma = 1e-3
    m = W.Surface("sag", "mirror", "circle", ap=(1.0, 0, 0, 0))
    scene = W.Scene("rough", [m], [W.Material([400.0], [1.0], sigma=sigma)], [W.Medium()], 1.0, 1.0)
    n = 100000
    r = _trace(scene, _bundle(np.tile([0.0, 0.0, 1.0], (n, 1)), [[0, 0, -1]] * n))
    dx, dy = r["dir"][0], r["dir"][1]
    for comp in (dx, dy):
        sd = comp.std()
        assert abs(sd / (2 * sigma) - 1.0) < 0.02
        assert abs(comp.mean()) < 5 * 2 * sigma / math.sqrt(n)
    assert abs(np.corrcoef(dx, dy)[0, 1]) < 0.02


def test_reflectivity_table_interpolation_and_clamping():
    mat = W.lst_reflectivity()
    assert oracle.reflectivity(mat, 300.0) == 0.85
    assert oracle.reflectivity(mat, 600.0) == 0.92
    assert abs(oracle.reflectivity(mat, 450.0) - 0.885) < 1e-15
    assert oracle.reflectivity(mat, 200.0) == 0.85 and oracle.reflectivity(mat, 900.0) == 0.92


def test_absorption_fraction_follows_reflectivity_table():
    mat = W.Material([300.0, 600.0], [0.5, 0.9])
    m = W.Surface("sag", "mirror", "circle", ap=(1.0, 0, 0, 0))
    scene = W.Scene("refl", [m], [mat], [W.Medium()], 1.0, 1.0)
    n = 40000
    for lam, R in ((300.0, 0.5), (450.0, 0.7), (600.0, 0.9)):
        r = _trace(scene, _bundle(np.tile([0.0, 0.0, 1.0], (n, 1)), [[0, 0, -1]] * n, lam=lam))
        surv = (r["status"] == ESCAPED).mean()
        assert abs(surv - R) < 5 * math.sqrt(R * (1 - R) / n)


def test_max_bounces_between_parallel_mirrors():
    lo = W.Surface("sag", "mirror", "circle", ap=(1.0, 0, 0, 0))
    hi = W.Surface("sag", "mirror", "circle", origin=(0, 0, 1.0), rot=W.FACING_DOWN, ap=(1.0, 0, 0, 0))
    scene = W.Scene("cavity", [lo, hi], [W.Material([400.0], [1.0])], [W.Medium()], 2.0, 1.0)
    r = _trace(scene, _bundle([[0.0, 0.0, 0.5]], [[1e-3, 0, -1]]), max_bounces=17)
    assert r["status"][0] == MAX_BOUNCES and r["bounces"][0] == 17


def test_back_side_hits_are_obscured():
    m = W.Surface("sag", "mirror", "circle", ap=(1.0, 0, 0, 0))
    scene = W.Scene("back", [m], [W.Material([400.0], [1.0])], [W.Medium()], 1.0, 1.0)
    r = _trace(scene, _bundle([[0.0, 0.0, -1.0]], [[0, 0, 1]]))
    assert r["status"][0] == OBSCURED and r["bounces"][0] == 1


# --------------------------------------------------------------- apertures
def test_hexagon_edges_are_inclusive():
    a = 0.5
    m = W.Surface("sag", "focal", "hexagon", ap=(a, 0, 0, 0))
    scene = W.Scene("hex", [m], [W.Material([400.0], [1.0])], [W.Medium()], 1.0, 1.0)
    s3 = math.sqrt(3.0)
    on_edge = [[a, 0.0], [-a, 0.1], [a * 0.5, a * s3 / 2], [0.0, a * 2 / s3]]  # flats and a corner
    out = [[a * (1 + 1e-12), 0.0], [0.0, a * 2 / s3 * (1 + 1e-12)]]
    pts = on_edge + out
    o = [[p[0], p[1], 1.0] for p in pts]
    r = _trace(scene, _bundle(o, [[0, 0, -1]] * len(o)))
    assert list(r["status"][:len(on_edge)]) == [DETECTED] * len(on_edge)
    assert list(r["status"][len(on_edge):]) == [ESCAPED] * len(out)


def test_sector_aperture_angles():
    m = W.Surface("sag", "focal", "sector", ap=(1.0, 2.0, math.radians(10), math.radians(40)))
    scene = W.Scene("sec", [m], [W.Material([400.0], [1.0])], [W.Medium()], 1.0, 1.0)
    tests = [(1.5, 25, True), (1.5, 9.9, False), (1.5, 40.1, False), (0.99, 25, False), (2.01, 25, False),
             (1.5, 205, False)]
    o = [[r * math.cos(math.radians(p)), r * math.sin(math.radians(p)), 1.0] for r, p, _ in tests]
    res = _trace(scene, _bundle(o, [[0, 0, -1]] * len(o)))
    assert [s == DETECTED for s in res["status"]] == [t[2] for t in tests]


def test_cylinder_mast_closed_form():
    """A ray crossing a vertical cylinder of radius a at impact parameter b
    enters at t = D - sqrt(a^2 - b^2)."""
    a = 0.1
    cyl = W.Surface("cylinder", "obscuration", prm=(a, 2.0, 0, 0, 0, 0, 0, 0))
    scene = W.Scene("cyl", [cyl], [W.Material([400.0], [1.0])], [W.Medium()], 3.0, 1.0)
    for bimp in (0.0, 0.05, 0.099):
        p = np.array([-1.0, bimp, 1.0])
        h = oracle.intersect(cyl, p, np.array([1.0, 0.0, 0.0]))
        assert abs(h[0] - (1.0 - math.sqrt(a * a - bimp * bimp))) < 1e-14
    r = _trace(scene, _bundle([[-1.0, 0.0, 1.0], [-1.0, 0.0, 2.5]], [[1, 0, 0], [1, 0, 0]]))
    assert list(r["status"]) == [OBSCURED, ESCAPED]


# ---------------------------------------------------------------- workloads
def test_lst_layout_has_198_facets_and_23m_aperture():
    c = W.lst_facet_centres()
    assert len(c) == 198
    rho = max(math.hypot(x, y) for x, y in c)
    assert 11.0 - 1e-9 <= rho + W.LST_PITCH / math.sqrt(3) <= 12.0


def test_sct_paraxial_focus():
    """Mirror equation for the two-mirror prescription: the secondary images
    the primary focus at z = 6.4 m, effective focal length 5.6 m."""
    f1 = W.SC_R1 / 2
    s = -(f1 - 8.4)
    s_img = 1 / (1 / (W.SC_R2 / 2) - 1 / s)
    assert abs(8.4 - s_img - 6.4) < 1e-12
    assert abs(f1 * s_img / abs(s) - 5.6) < 1e-12


def test_gct_paraxial_focus_by_mirror_equation_and_trace():
    """GCT-like prescription: the mirror equation puts the secondary's image of
    the primary focus at the focal surface's vertex z = 6.4 s with effective
    focal length 2.283 m; tracing near-axis rays through the two mirrors
    (apertures opened, asphere terms off: the paraxial system) reproduces both:
    a ray at height h leaves the secondary at angle atan(h / EFL) and crosses
    the axis at the image point."""
    s = W.GCT_S
    R1, R2 = W.SC_R1 * s, W.SC_R2 * s
    f1 = R1 / 2
    z2 = 8.4 * s
    so = -(f1 - z2)
    si = 1 / (1 / (R2 / 2) - 1 / so)
    assert abs(z2 - si - 6.4 * s) < 1e-12
    assert abs(f1 * si / abs(so) - W.GCT_F) < 1e-12
    prim = W.Surface("sag", "mirror", "circle", curv=1.0 / R1, ap=(4.85 * s, 0, 0, 0))
    sec = W.Surface("sag", "mirror", "circle", origin=(0.0, 0.0, z2), rot=W.FACING_DOWN, curv=1.0 / R2,
                    ap=(2.7 * s, 0, 0, 0))
    scene = W.Scene("gct_paraxial", [prim, sec], [W.Material([400.0], [1.0])], [W.Medium()], 7.0, W.GCT_F)
    hs = np.array([1e-4, 2e-4, 5e-4])
    phi = np.array([0.3, 1.7, 4.0])
    o = np.stack([hs * np.cos(phi), hs * np.sin(phi), np.full(3, z2 - 0.01)])
    b = W.Bundle(o, np.repeat([[0.0], [0.0], [-1.0]], 3, axis=1), np.full(3, 400.0))
    r = _trace(scene, b, max_bounces=2)  # stop after the secondary: the last point is on it
    assert np.all(r["status"] == MAX_BOUNCES) and np.all(r["last_surface"] == 1)
    d = r["dir"]
    p = r["hit"]
    rho_d = np.hypot(d[0], d[1])
    efl = hs * (-d[2]) / rho_d
    assert np.max(np.abs(efl / W.GCT_F - 1)) < 1e-6
    # axis crossing of the outgoing line through the last point, along the radial direction
    radial = (p[0] * np.cos(phi) + p[1] * np.sin(phi))
    drad = d[0] * np.cos(phi) + d[1] * np.sin(phi)
    zc = p[2] - radial * d[2] / drad
    assert np.max(np.abs(zc - 6.4 * s)) < 1e-6


def test_gct_scene_detects_through_both_mirrors():
    scene, b = W.gct_workload(4_000, seed=2)
    s = W.GCT_S
    mirrors = [x for x in scene.surfaces if x.role == "mirror"]
    assert len(mirrors) == 7  # six primary petals, one secondary
    assert all(abs(m.curv - 1 / (W.SC_R1 * s)) < 1e-15 and m.origin[2] == 0.0 for m in mirrors[:6])
    assert abs(mirrors[6].curv - 1 / (W.SC_R2 * s)) < 1e-15 and abs(mirrors[6].origin[2] - 8.4 * s) < 1e-15
    assert abs(scene.surfaces[0].origin[2] - 6.4 * s) < 1e-15
    r = _trace(scene, b)
    det = r["status"] == DETECTED
    assert det.mean() > 0.3
    assert np.all(r["bounces"][det] == 3)
    # detected photons last met the focal surface (surface 0) after a petal and the secondary
    assert np.all(r["last_surface"][det] == 0)
