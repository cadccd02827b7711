"""Pins of the oracle's source generator (uniform points on a hexagon)."""
import math

import numpy as np

import oracle


def _gen(n, seed=1, apothem=0.025):
    b, v, failed = oracle.generate_sources(
        [dict(variant=2, n=n, centre=(0.01, -0.02, 0.07), apothem=apothem, dir=(0.6, 0.0, -0.8), lam=(300, 600))],
        seed=seed)
    return b, v, failed


def test_points_inside_hexagon_plane_and_direction():
    b, v, failed = _gen(50_000)
    assert failed == 0
    x = b["origins"][0] - 0.01
    y = b["origins"][1] + 0.02
    s = math.sqrt(3) / 2
    m = np.maximum.reduce([np.abs(x), np.abs(0.5 * x + s * y), np.abs(-0.5 * x + s * y)])
    assert np.all(m <= 0.025)
    assert np.all(b["origins"][2] == 0.07)
    assert np.all(b["dirs"][0] == 0.6) and np.all(b["dirs"][2] == -0.8)
    assert np.all(v == 2)


def test_uniform_over_the_hexagon():
    """Counts in the six triangles and in a central disk follow the areas."""
    n = 200_000
    b, _, _ = _gen(n, seed=4, apothem=1.0)
    x = b["origins"][0] - 0.01
    y = b["origins"][1] + 0.02
    sector = np.floor(((np.arctan2(y, x) + np.pi / 6) % (2 * np.pi)) / (np.pi / 3)).astype(int)
    counts = np.bincount(sector, minlength=6)
    exp = n / 6
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 5 + 6 * math.sqrt(10)  # 5 dof
    area = 2 * math.sqrt(3)  # hexagon of apothem 1
    p = math.pi * 0.5 ** 2 / area
    k = (np.hypot(x, y) <= 0.5).sum()
    assert abs(k / n - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_wavelength_uniform_and_ids_matter():
    b, _, _ = _gen(100_000, seed=7)
    lam = b["wavelengths"]
    assert lam.min() >= 300 and lam.max() <= 600
    assert abs(lam.mean() - 450) < 5 * 300 / math.sqrt(12 * 100_000)
    b2, _, _ = _gen(100_000, seed=8)
    assert not np.array_equal(b["origins"], b2["origins"])
    b3, _, _ = oracle.generate_sources([dict(variant=0, n=10, centre=(0, 0, 0), apothem=1.0, dir=(0, 0, -1),
                                             lam=(300, 600))], seed=7, first_photon_id=5)
    b4, _, _ = oracle.generate_sources([dict(variant=0, n=15, centre=(0, 0, 0), apothem=1.0, dir=(0, 0, -1),
                                             lam=(300, 600))], seed=7)
    assert np.array_equal(b3["origins"], b4["origins"][:, 5:])
