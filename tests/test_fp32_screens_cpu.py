"""Three FP32 shortcuts of the CUDA path, checked numerically on the CPU.

1. The spot-diagram reduction bins r^2 in FP32 (dx = x - fl(cx), r2 =
   fma(dx, dx, fl(dy * dy)), f = fl(r2 * fl(scale))) and trusts the bin only
   where its error bound delta (computed per window from the centroid and the
   range) is below 1/2.  Here every photon's |f_FP32 - f_exact| must stay
   below delta, on spots placed to stress the bound.
2. The device photon source screens each hexagon candidate in FP32 and
   decides in FP64 only within 1e-5 a of the boundary; the FP32 hexagon
   measure must stay within 2e-6 a of the FP64 one.
3. The FP64 nearest-hit search screens each sag candidate in FP32 (rebased
   in FP32 from float pairs) before its FP64 test; a ray the screen excludes
   must have no hit in the oracle's FP64 intersection of that surface, for
   aspheric SC panels and for tilted dish facets far from the origin; the
   same for the cylinder screen on the dish's slanted masts.

numpy float32 arithmetic rounds once per operation, as the device does; the
fused multiply-add is emulated exactly (the product of two floats is exact in
FP64, then one rounding to FP32).
"""
import math

import numpy as np

F = np.float32
K_BINS = 4096


def fmaf(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def delta_bound(cx, cy, scale):
    """The bound of the reduction's finish step, restated from its derivation."""
    u = 2.0 ** -24
    R2 = (K_BINS + 2) / scale
    R = math.sqrt(R2)
    ex = u * abs(cx) * (1 + u) + u * R
    ey = u * abs(cy) * (1 + u) + u * R
    E = R + ex + ey
    err = ex * (2 * R + ex) + ey * (2 * R + ey) + (2 * u + u * u) * E * E
    return scale * err + (2 * u + u * u) * scale * (R2 + err)


def test_fp32_binning_error_stays_below_the_bound():
    rng = np.random.default_rng(5)
    cases = [((0.3, -1.02), 0.02), ((0.0, 0.0), 0.03), ((-1.5, 2.0), 0.005), ((1.0, 1.0), 1e-4), ((12.0, -7.0), 0.05)]
    for (mx, my), sig in cases:
        x = (rng.normal(mx, sig, 400_000)).astype(F)
        y = (rng.normal(my, sig, 400_000)).astype(F)
        xd, yd = x.astype(np.float64), y.astype(np.float64)
        cx, cy = xd.mean(), yd.mean()
        ms = ((xd - cx) ** 2 + (yd - cy) ** 2).mean()
        scale = K_BINS / (64.0 * ms)
        delta = delta_bound(cx, cy, scale)
        dx = (x - F(cx)).astype(F)
        dy = (y - F(cy)).astype(F)
        r2f = fmaf(dx, dx, (dy * dy).astype(F))
        ff = (r2f * F(scale)).astype(F).astype(np.float64)
        fe = ((xd - cx) ** 2 + (yd - cy) ** 2) * scale  # exact to FP64 rounding
        inside = fe < K_BINS + 2
        err = np.max(np.abs(ff[inside] - fe[inside]))
        assert err <= delta, ((mx, my), sig, err, delta)
        if delta < 0.1:  # the bound is not vacuous where the fast path is used
            assert err > 0.0


def test_fp32_hexagon_screen_stays_within_its_band():
    rng = np.random.default_rng(9)
    n = 2_000_000
    for a in (0.025, 1.0, 12.0):
        R = a * 2.0 / math.sqrt(3.0)
        w0 = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
        w1 = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
        # FP64 definition
        u0 = (w0.astype(np.float64) + 0.5) * 2.0 ** -32
        u1 = (w1.astype(np.float64) + 0.5) * 2.0 ** -32
        x = (2.0 * u0 - 1.0) * a
        y = (2.0 * u1 - 1.0) * R
        s60 = 0.86602540378443864676
        m64 = np.maximum(np.abs(x), np.maximum(np.abs(0.5 * x + s60 * y), np.abs(-0.5 * x + s60 * y)))
        # FP32 screen, one rounding per operation (fused forms are at least as accurate)
        u0f = ((w0.astype(F) + F(0.5)) * F(2.0 ** -32)).astype(F)
        u1f = ((w1.astype(F) + F(0.5)) * F(2.0 ** -32)).astype(F)
        xf = ((F(2.0) * u0f - F(1.0)) * F(a)).astype(F)
        yf = ((F(2.0) * u1f - F(1.0)) * F(R)).astype(F)
        hx, sy = (F(0.5) * xf).astype(F), (F(s60) * yf).astype(F)
        mf = np.maximum(np.abs(xf), np.maximum(np.abs(hx + sy), np.abs(sy - hx))).astype(np.float64)
        assert np.max(np.abs(mf - m64)) <= 2e-6 * a, a
        # the screen never decides against the FP64 test outside its band
        a32 = float(F(a))
        sure_in = mf < a32 * float(F(1.0) - F(1e-5))
        sure_out = mf > a32 * float(F(1.0) + F(1e-5))
        assert np.all(m64[sure_in] <= a) and np.all(m64[sure_out] > a)


def _aperture_near_sector(ap32, x, y, m):
    """The FP64 search's aperture test with margin m for an annular sector (FP32 record values)."""
    rmin, rmax, c0, s0, c1, s1 = ap32
    r = np.sqrt((x * x + y * y).astype(F)).astype(F)
    return (r >= rmin - m) & (r <= rmax + m) & ((c0 * y - s0 * x).astype(F) >= -m) & ((x * s1 - y * c1).astype(F) >= -m)


def _screen_asph_may_hit(c, k1, rb2, adev, ap32, p, d, eps):
    """The FP32 screen of an aspheric candidate (device `screen_asph_miss`), restated with one
    FP32 rounding per operation: True where the candidate must go to the FP64 test."""
    c, k1 = F(c), F(k1)
    px, py, pz = (p[k].astype(F) for k in range(3))
    dx, dy, dz = (d[k].astype(F) for k in range(3))
    ac, ak = F(abs(c)), F(abs(k1))
    mp = (np.abs(px) + np.abs(py) + np.abs(pz)).astype(F)
    a = (c * (dx * dx + dy * dy + k1 * dz * dz)).astype(F)
    b = (c * (px * dx + py * dy + k1 * pz * dz) - dz).astype(F)
    g = (c * (px * px + py * py + k1 * pz * pz) - F(2) * pz).astype(F)
    aa = (ac * (dx * dx + dy * dy + ak * dz * dz)).astype(F)
    bb = (ac * (np.abs(px * dx) + np.abs(py * dy) + ak * np.abs(pz * dz)) + np.abs(dz)).astype(F)
    gg = (ac * (px * px + py * py + ak * pz * pz) + F(2) * np.abs(pz)).astype(F)
    may = np.zeros(px.shape, bool)
    open_ = np.ones(px.shape, bool)  # not decided yet

    def decide(mask, value):
        nonlocal may, open_
        mask = mask & open_
        may[mask] = value[mask] if isinstance(value, np.ndarray) else value
        open_ &= ~mask

    decide(~(np.abs(a) > F(1e-2) * aa) | ~(np.abs(b) > F(1e-2) * bb) | ~(np.abs(g) > F(1e-2) * gg), True)
    disc = (b * b - a * g).astype(F)
    decide(~(np.abs(disc) > F(1e-2) * (b * b + np.abs(a * g))), True)
    decide(disc < 0, False)
    with np.errstate(all="ignore"):
        sq = np.sqrt(np.maximum(disc, F(0))).astype(F)
        qq = (-(b + np.copysign(sq, b))).astype(F)
        t1, t2 = (qq / a).astype(F), (g / qq).astype(F)
    tl, th = np.minimum(t1, t2), np.maximum(t1, t2)
    decide(~((th - tl) > F(2e-3) * (np.abs(tl) + np.abs(th) + mp)), True)
    ep = F(eps)
    for t in (tl, th):
        mt = (F(1e-3) * (np.abs(t) + mp)).astype(F)
        qx, qy, qz = (px + t * dx).astype(F), (py + t * dy).astype(F), (pz + t * dz).astype(F)
        v = (k1 * c * qz - F(1)).astype(F)
        mv = (F(1e-2) + ac * ak * mt).astype(F)
        skip = open_ & (v > mv)
        decide(~skip & ~(v < -mv), True)
        skip |= open_ & (t < ep - mt)
        decide(~skip & ~(t > ep + mt), True)
        here = open_ & ~skip  # the first qualifying root
        eq = (mt + F(1e-3) * (np.abs(qx) + np.abs(qy))).astype(F)
        r = np.sqrt(qx * qx + qy * qy).astype(F)
        rb = F(math.sqrt(float(F(rb2))))
        decide(here & (r > rb * F(1.001) + eq), False)
        decide(here & ~(r < rb * F(0.999) - eq), True)
        mx, my, mz = (-c * qx).astype(F), (-c * qy).astype(F), (F(1) - c * k1 * qz).astype(F)
        nn = (mx * mx + my * my + mz * mz).astype(F)
        dn = np.abs(dx * mx + dy * my + dz * mz).astype(F)
        decide(here & ~(dn * dn > F(0.0025) * F(1.01) * nn), True)
        with np.errstate(all="ignore"):
            m = (F(2) * F(adev) * np.sqrt(nn) / dn + F(1e-4) * (np.abs(qx) + np.abs(qy) + np.abs(t))).astype(F)
        decide(here, _aperture_near_sector(ap32, qx, qy, (F(1.001) * m + eq).astype(F)))
    decide(np.ones(px.shape, bool), False)  # no qualifying root
    return may


def test_fp32_asphere_screen_never_rejects_a_hit():
    """The FP64 search screens each aspheric candidate in FP32 first and skips the FP64 test
    where the screen excludes a hit.  On rays aimed at and around an aspheric SC primary panel
    (from above, obliquely, grazing, from below), every ray the screen excludes must have no hit
    in the oracle's FP64 intersection of that panel (nor a Newton failure, which the FP64 test
    reports), and the screen must exclude most rays that miss (it is not vacuous)."""
    import oracle
    import workloads as W
    scene = W.sct_scene(seed=0)
    L = scene.length_scale
    eps = 1e-9 * L
    rng = np.random.default_rng(17)
    for idx in (2, 20):  # an inner-ring and an outer-ring primary panel (identity frame at the origin)
        s = scene.surfaces[idx]
        assert s.shape == "sag" and any(a != 0 for a in s.asph)
        rmin, rmax, phi0, phi1 = s.ap[:4]
        rb = 1.1 * rmax
        rb2 = rb * rb
        adev = sum(abs(s.asph[k]) * rb2 ** (k + 1) for k in range(8))
        ap32 = tuple(F(v) for v in (rmin, rmax, math.cos(phi0), math.sin(phi0), math.cos(phi1), math.sin(phi1)))
        n = 6000
        rows = []
        # from above towards points around the panel, some nearly parallel to the mirror
        for zt_lo, zt_hi, z0_lo, z0_hi in ((0.0, 0.6, 4.0, 14.0), (0.0, 0.6, 0.3, 1.2), (-1.0, 1.0, -3.0, -0.5)):
            tx = rng.uniform(-6.0, 6.0, n)
            ty = rng.uniform(-6.0, 6.0, n)
            tz = rng.uniform(zt_lo, zt_hi, n)
            ox = rng.uniform(-8.0, 8.0, n)
            oy = rng.uniform(-8.0, 8.0, n)
            oz = rng.uniform(z0_lo, z0_hi, n)
            dd = np.stack([tx - ox, ty - oy, tz - oz])
            dd /= np.linalg.norm(dd, axis=0)
            rows.append((np.stack([ox, oy, oz]), dd))
        # aimed at the panel's sector and just beyond its edges, from above and obliquely
        rr = rng.uniform(rmin - 0.2, rmax + 0.2, 2 * n)
        ph = rng.uniform(phi0 - 0.1, phi1 + 0.1, 2 * n)
        tgt = np.stack([rr * np.cos(ph), rr * np.sin(ph), rng.uniform(0.0, 0.6, 2 * n)])
        org = tgt + np.stack([rng.uniform(-6.0, 6.0, 2 * n), rng.uniform(-6.0, 6.0, 2 * n),
                              rng.uniform(0.5, 12.0, 2 * n)])
        dd = tgt - org
        dd /= np.linalg.norm(dd, axis=0)
        rows.append((org, dd))
        p = np.concatenate([r[0] for r in rows], axis=1)
        d = np.concatenate([r[1] for r in rows], axis=1)
        p32 = p.astype(F).astype(np.float64)
        d32 = d.astype(F).astype(np.float64)
        may = _screen_asph_may_hit(s.curv, 1.0 + s.conic, rb2, adev, ap32, p32, d32, eps)
        def fp64_needed(i):  # a hit, or a Newton failure (which the FP64 test reports as ERROR)
            try:
                return oracle.intersect(s, p32[:, i], d32[:, i], eps) is not None
            except ArithmeticError:
                return True

        hits = np.array([fp64_needed(i) for i in range(p.shape[1])])
        assert not np.any(hits & ~may), f"panel {idx}: the screen excluded {int((hits & ~may).sum())} hits"
        assert hits.sum() > 2000
        assert (~may).sum() > 0.5 * (~hits).sum(), f"panel {idx}: the screen excluded only {int((~may).sum())} rays"


def _rows_tilted(s):
    """The facet's tilted frame rows, Ry(b)^T Rx(a)^T R (rows = local axes in world coordinates)."""
    ca, sa = math.cos(s.tilt[0]), math.sin(s.tilt[0])
    cb, sb = math.cos(s.tilt[1]), math.sin(s.tilt[1])
    rxT = np.array([[1, 0, 0], [0, ca, sa], [0, -sa, ca]])
    ryT = np.array([[cb, 0, -sb], [0, 1, 0], [sb, 0, cb]])
    return ryT @ (rxT @ np.asarray(s.rot, np.float64).reshape(3, 3))


def _rebase32(rows, origin, p, d):
    """The FP64 search's FP32 rebase: the photon as a float pair minus the origin as a float pair,
    then the FP32 rows; one FP32 rounding per operation."""
    o = np.asarray(origin, np.float64)
    ohi = o.astype(F)
    olo = (o - ohi.astype(np.float64)).astype(F)
    phi = p.astype(F)
    plo = (p - phi.astype(np.float64)).astype(F)
    q = ((phi - ohi[:, None]).astype(F) + (plo - olo[:, None]).astype(F)).astype(F)
    R = rows.astype(F)
    d32 = d.astype(F)

    def rot(v):
        return np.stack([((R[k, 0] * v[0]).astype(F) + (R[k, 1] * v[1]).astype(F) + (R[k, 2] * v[2]).astype(F))
                         .astype(F) for k in range(3)])

    return rot(q), rot(d32)


def _screen_sag_may_hit(c, k1, apothem, p, d, eps):
    """The FP32 screen of a sag candidate without asphere terms (device `screen_sag_miss`, no best
    hit yet, hexagonal aperture), restated with one FP32 rounding per operation."""
    c, k1 = F(c), F(k1)
    px, py, pz = p
    dx, dy, dz = d
    ac, ak = F(abs(c)), F(abs(k1))
    mp = (np.abs(px) + np.abs(py) + np.abs(pz)).astype(F)
    a = (c * (dx * dx + dy * dy + k1 * dz * dz)).astype(F)
    b = (c * (px * dx + py * dy + k1 * pz * dz) - dz).astype(F)
    g = (c * (px * px + py * py + k1 * pz * pz) - F(2) * pz).astype(F)
    aa = (ac * (dx * dx + dy * dy + ak * dz * dz)).astype(F)
    bb = (ac * (np.abs(px * dx) + np.abs(py * dy) + ak * np.abs(pz * dz)) + np.abs(dz)).astype(F)
    gg = (ac * (px * px + py * py + ak * pz * pz) + F(2) * np.abs(pz)).astype(F)
    ill = ~(np.abs(a) > F(1e-2) * aa) | ~(np.abs(b) > F(1e-2) * bb) | ~(np.abs(g) > F(1e-2) * gg)
    disc = (b * b - a * g).astype(F)
    ill |= ~(np.abs(disc) > F(1e-2) * (b * b + np.abs(a * g)))
    with np.errstate(all="ignore"):
        sq = np.sqrt(np.maximum(disc, F(0))).astype(F)
        qq = (-(b + np.copysign(sq, b))).astype(F)
        roots = ((qq / a).astype(F), (g / qq).astype(F))
    may = np.zeros(px.shape, bool)
    s60 = F(0.86602540378443864676)
    for t in roots:
        mt = (F(1e-3) * (np.abs(t) + mp)).astype(F)
        ok = (t > F(eps) - mt) & (t < F(3.0e38) + mt)
        qx, qy, qz = (px + t * dx).astype(F), (py + t * dy).astype(F), (pz + t * dz).astype(F)
        ok &= ~((k1 * c * qz - F(1)).astype(F) > F(1e-2) + ac * ak * mt)
        h = np.maximum(np.abs(qx), np.maximum(np.abs(F(0.5) * qx + s60 * qy), np.abs(F(-0.5) * qx + s60 * qy)))
        ok &= h <= F(apothem) + (mt + F(1e-3) * (np.abs(qx) + np.abs(qy))).astype(F)
        may |= ok
    return ill | (~(disc < 0) & may)


def test_fp32_rebase_and_sag_screen_never_reject_a_hit():
    """The FP64 search rebases each sag candidate in FP32 (photon and origin as float pairs, FP32
    frame rows) and screens it before any FP64 instruction.  On dish facets far from the origin,
    with tilted frames, rays coming down from the source plane and going up from the dish must
    never be excluded where the oracle's FP64 intersection hits, and most misses must be."""
    import oracle
    import workloads as W
    scene = W.lst_scene(seed=0)
    eps = 1e-9 * scene.length_scale
    rng = np.random.default_rng(23)
    facets = [s for s in scene.surfaces if s.shape == "sag" and s.role == "mirror"]
    for s in (facets[0], facets[97], facets[-1]):
        c = np.asarray(s.origin)
        n = 8000
        # down from the source plane towards points within 3 m of the facet centre
        tgt = c[:, None] + np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-0.3, 0.3, n)])
        org = np.stack([tgt[0] + rng.uniform(-1, 1, n), tgt[1] + rng.uniform(-1, 1, n), np.full(n, 32.0)])
        # up from points near the facet towards the focal plane
        org2 = c[:, None] + np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(-0.2, 0.5, n)])
        tgt2 = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n), np.full(n, 28.0)])
        p = np.concatenate([org, org2], axis=1)
        d = np.concatenate([tgt - org, tgt2 - org2], axis=1)
        d /= np.linalg.norm(d, axis=0)
        p32 = p.astype(F).astype(np.float64)
        d32 = d.astype(F).astype(np.float64)
        pl, dl = _rebase32(_rows_tilted(s), s.origin, p32, d32)
        may = _screen_sag_may_hit(s.curv, 1.0 + s.conic, s.ap[0], pl, dl, eps)
        hits = np.array([oracle.intersect(s, p32[:, i], d32[:, i], eps) is not None for i in range(p.shape[1])])
        assert not np.any(hits & ~may), f"the screen excluded {int((hits & ~may).sum())} hits"
        assert hits.sum() > 500
        assert (~may).sum() > 0.5 * (~hits).sum()


def _screen_cyl_may_hit(rad, length, p, d, eps):
    """The FP32 screen of a cylinder candidate (device `screen_cyl_miss`, no best hit yet),
    restated with one FP32 rounding per operation."""
    rad, length = F(rad), F(length)
    px, py, pz = p
    dx, dy, dz = d
    a = (dx * dx + dy * dy).astype(F)
    near_axis = ~(a >= F(1e-2) * (a + dz * dz))
    with np.errstate(all="ignore"):
        t0 = (-(px * dx + py * dy) / a).astype(F)
        cx, cy = (px + t0 * dx).astype(F), (py + t0 * dy).astype(F)
        m = (F(1e-3) * (np.abs(px) + np.abs(py) + np.abs(pz) + np.abs(t0))).astype(F)
        dist = np.sqrt(cx * cx + cy * cy).astype(F)
        H = ((rad + m) / np.sqrt(a)).astype(F)
    tlo, thi = (t0 - H).astype(F), (t0 + H).astype(F)
    mt = (m + F(1e-3) * H).astype(F)
    z0, z1 = (pz + tlo * dz).astype(F), (pz + thi * dz).astype(F)
    miss = (dist > rad + m) | (thi < F(eps) - mt) | (tlo > F(3.0e38) + mt) | \
           (np.maximum(z0, z1) < -mt) | (np.minimum(z0, z1) > length + mt)
    return near_axis | ~miss


def test_fp32_rebase_and_cylinder_screen_never_reject_a_hit():
    """The same for the dish's slanted masts (cylinders in tilted frames from the rim to the
    camera box): rays from the source plane and from the dish must never be excluded where the
    oracle's FP64 intersection hits, and most misses must be."""
    import oracle
    import workloads as W
    scene = W.lst_scene(seed=0)
    eps = 1e-9 * scene.length_scale
    rng = np.random.default_rng(29)
    masts = [s for s in scene.surfaces if s.shape == "cylinder"]
    assert len(masts) == 4
    for s in masts[:2]:
        o = np.asarray(s.origin)
        axis = _rows_tilted(s)[2]
        n = 8000
        # targets along the mast and up to 0.5 m off it
        tt = rng.uniform(-1.0, s.prm[1] + 1.0, n)
        tgt = o[:, None] + axis[:, None] * tt + rng.uniform(-0.5, 0.5, (3, n))
        org = np.concatenate([np.stack([tgt[0, :n // 2] + rng.uniform(-2, 2, n // 2),
                                        tgt[1, :n // 2] + rng.uniform(-2, 2, n // 2), np.full(n // 2, 32.0)]),
                              np.stack([rng.uniform(-11, 11, n - n // 2), rng.uniform(-11, 11, n - n // 2),
                                        rng.uniform(0.0, 1.2, n - n // 2)])], axis=1)
        d = tgt - org
        d /= np.linalg.norm(d, axis=0)
        p32 = org.astype(F).astype(np.float64)
        d32 = d.astype(F).astype(np.float64)
        pl, dl = _rebase32(_rows_tilted(s), s.origin, p32, d32)
        may = _screen_cyl_may_hit(s.prm[0], s.prm[1], pl, dl, eps)
        hits = np.array([oracle.intersect(s, p32[:, i], d32[:, i], eps) is not None for i in range(n)])
        assert not np.any(hits & ~may), f"the screen excluded {int((hits & ~may).sum())} hits"
        assert hits.sum() > 300
        assert (~may).sum() > 0.5 * (~hits).sum()
