"""Pins of refraction beyond a window: bulk absorption (Beer-Lambert) and a
thick lens (paraxial back focal distance from the lensmaker's equation)."""
import math

import numpy as np

import oracle
import workloads as W


def _bundle(o, d, lam=400.0):
    o = np.ascontiguousarray(np.asarray(o, np.float64).T)
    d = np.asarray(d, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return W.Bundle(o, np.ascontiguousarray(d.T), np.full(o.shape[1], float(lam)))


def test_absorption_length_table():
    m = W.Medium(n_const=1.5, abs_lam=(300.0, 500.0), abs_len=(0.01, 0.05))
    assert oracle.lib().oracle_absorption_length(oracle.pack_medium(m), 300.0) == 0.01
    assert abs(oracle.lib().oracle_absorption_length(oracle.pack_medium(m), 400.0) - 0.03) < 1e-15
    assert oracle.lib().oracle_absorption_length(oracle.pack_medium(m), 900.0) == 0.05
    assert math.isinf(oracle.lib().oracle_absorption_length(oracle.pack_medium(W.Medium()), 400.0))


def test_beer_lambert_through_an_index_matched_slab():
    """n = 1 on both sides: no refraction, no Fresnel loss; the slab only
    absorbs, so the transmitted fraction is exp(-T / (L cos theta))."""
    T, L = 0.01, 0.02
    top = W.Surface("sag", "refract", "circle", origin=(0, 0, T), medium_front=0, medium_back=1, ap=(1.0, 0, 0, 0))
    bot = W.Surface("sag", "refract", "circle", origin=(0, 0, 0), medium_front=1, medium_back=0, ap=(1.0, 0, 0, 0))
    scene = W.Scene("slab", [top, bot], [W.Material([400.0], [1.0])],
                    [W.Medium(), W.Medium(n_const=1.0, abs_lam=(400.0,), abs_len=(L,))], 1.0, 1.0)
    n = 40_000
    for theta in (0.0, 0.6):
        d = [[math.sin(theta), 0.0, -math.cos(theta)]] * n
        r = oracle.trace(scene, _bundle(np.tile([0.0, 0.0, 0.05], (n, 1)), d), n_threads=4)
        through = ((r["status"] == W.ESCAPED) & (r["bounces"] == 2)).mean()
        p = math.exp(-T / (L * math.cos(theta)))
        assert abs(through - p) < 5 * math.sqrt(p * (1 - p) / n)
        assert np.all(np.isin(r["status"], [W.ESCAPED, W.ABSORBED]))


def test_plano_convex_lens_paraxial_back_focal_distance():
    """Lensmaker: f = R / (n - 1) for a plano-convex lens; the back focal
    distance behind the flat face is f - T / n.  Paraxial rays cross the axis
    there up to spherical aberration, which falls as h^2."""
    R, T, n = 0.1, 0.01, 1.49
    scene = W.lens_scene(R1=R, thickness=T, n=n)
    f = R / (n - 1)
    bfd = f - T / n
    errs = []
    for h in (4e-4, 2e-4, 1e-4):
        m = 64
        o = np.tile([h, 0.0, 0.05], (m, 1))
        r = oracle.trace(scene, _bundle(o, [[0.0, 0.0, -1.0]] * m), n_threads=2)
        ok = (r["status"] == W.ESCAPED) & (r["bounces"] == 2) & (r["dir"][2] < 0)
        assert ok.any()
        i = np.where(ok)[0][0]
        xe, ze = r["hit"][0][i], r["hit"][2][i]
        dx, dz = r["dir"][0][i], r["dir"][2][i]
        z_cross = ze + (-xe / dx) * dz
        errs.append(abs(-z_cross - bfd))
    # spherical aberration: error ~ h^2 (ratio ~4 per halving) and small at h = 1e-4
    assert errs[2] < 1e-6 * f
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
