"""Seeded synthetic workloads: optical-system descriptions and photon bundles.

This module is input generation only.  It builds the optical systems the
paper applies its tracer to (Sec. 3: a segmented parabolic dish with masts and
a camera box, Schwarzschild-Couder aspheric two-mirror optics, hexagonal
Winston / Bezier light concentrators) as plain Python records, and it draws
photon bundles from numpy's Philox4x64 generator.  It contains none of the
trace arithmetic (intersections, interactions, random streams of the trace):
both the CUDA library and the CPU oracle consume what it produces, each
through its own binding.

Units: metres, nanometres for wavelengths, radians for angles.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SHAPES = ("sag", "cylinder", "box", "hexcone")
ROLES = ("mirror", "refract", "focal", "obscuration")
APERTURES = ("none", "circle", "annulus", "sector", "hexagon", "rect")

STATUS_NAMES = {1: "DETECTED", 2: "ABSORBED", 3: "OBSCURED", 4: "ESCAPED", 5: "MAX_BOUNCES", 6: "ERROR"}
DETECTED, ABSORBED, OBSCURED, ESCAPED, MAX_BOUNCES, ERROR = 1, 2, 3, 4, 5, 6


@dataclasses.dataclass
class Surface:
    shape: str
    role: str
    aperture: str = "none"
    material: int = 0
    medium_front: int = 0
    medium_back: int = 0
    origin: Sequence[float] = (0.0, 0.0, 0.0)
    rot: Sequence[float] = (1, 0, 0, 0, 1, 0, 0, 0, 1)  # rows = local axes in world coords
    tilt: Sequence[float] = (0.0, 0.0)
    curv: float = 0.0
    conic: float = 0.0
    asph: Sequence[float] = (0.0,) * 8
    ap: Sequence[float] = (0.0,) * 4
    prm: Sequence[float] = (0.0,) * 8


@dataclasses.dataclass
class Material:
    lam: Sequence[float]
    refl: Sequence[float]
    sigma: float = 0.0


@dataclasses.dataclass
class Medium:
    n_const: float = 1.0
    B: Sequence[float] = (0.0, 0.0, 0.0)
    C: Sequence[float] = (0.0, 0.0, 0.0)
    abs_lam: Sequence[float] = ()  # bulk absorption: wavelengths (nm) of the table, empty = none
    abs_len: Sequence[float] = ()  # absorption lengths (m) at abs_lam


@dataclasses.dataclass
class Scene:
    name: str
    surfaces: List[Surface]
    materials: List[Material]
    media: List[Medium]
    length_scale: float  # L_sys: sets the self-intersection epsilon
    focal_length: float  # position tolerances are quoted relative to it
    variant_offsets: Optional[List[int]] = None

    @property
    def n_variants(self) -> int:
        return 1 if self.variant_offsets is None else len(self.variant_offsets) - 1


def _pad(seq, n):
    out = list(seq) + [0.0] * (n - len(seq))
    return out[:n]


def frame_from_axis(zaxis, xref=(1.0, 0.0, 0.0)):
    """Rows (x, y, z) of a right-handed frame whose z is `zaxis` and whose x is
    the projection of `xref` on the plane normal to z."""
    z = np.asarray(zaxis, dtype=np.float64)
    z = z / np.linalg.norm(z)
    xr = np.asarray(xref, dtype=np.float64)
    x = xr - np.dot(xr, z) * z
    if np.linalg.norm(x) < 1e-12:
        xr = np.array([0.0, 1.0, 0.0])
        x = xr - np.dot(xr, z) * z
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    return tuple(np.concatenate([x, y, z]).tolist())


FACING_DOWN = (1.0, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0, 0.0, -1.0)  # local z = world -z


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


# ----------------------------------------------------------------- scenes
def sphere_scene() -> Scene:
    """Single spherical mirror: R = 10 m (f = 5 m), circular aperture 1.0 m,
    reflectivity 0.9, no roughness; 0.3 m square focal plane at z = 5 m facing
    the mirror (its back shadows the incoming bundle)."""
    mat = Material(lam=[400.0], refl=[0.9], sigma=0.0)
    mirror = Surface("sag", "mirror", "circle", material=0, curv=1.0 / 10.0, ap=(0.5, 0, 0, 0))
    focal = Surface("sag", "focal", "rect", origin=(0.0, 0.0, 5.0), rot=FACING_DOWN, ap=(0.15, 0.15, 0, 0))
    return Scene("sphere", [mirror, focal], [mat], [Medium()], length_scale=10.0, focal_length=5.0)


LST_F = 28.0
LST_PITCH = 1.51
LST_CUT = 11.0


def lst_facet_centres(n_max: Optional[int] = None):
    """Hexagonal lattice (pitch 1.51 m, basis (1,0), (1/2, sqrt3/2)), centres
    with 0 < rho <= 11.0 m: 198 of them, ordered by radius then azimuth."""
    pts = []
    m = int(LST_CUT / LST_PITCH) + 3
    for i in range(-2 * m, 2 * m + 1):
        for j in range(-2 * m, 2 * m + 1):
            x = (i + 0.5 * j) * LST_PITCH
            y = (math.sqrt(3.0) / 2.0) * j * LST_PITCH
            rho = math.hypot(x, y)
            if 0.0 < rho <= LST_CUT:
                pts.append((round(rho, 9), math.atan2(y, x) % (2 * math.pi), x, y))
    pts.sort()
    pts = [(p[2], p[3]) for p in pts]
    if n_max is not None:
        pts = pts[:n_max]
    return pts


def lst_reflectivity() -> Material:
    return Material(lam=[300.0, 600.0], refl=[0.85, 0.92], sigma=0.3e-3)


def lst_scene(tilt_sigma: float = 0.1e-3, seed: int = 0, n_facets: Optional[int] = None,
              roughness: float = 0.3e-3, with_structure: bool = True) -> Scene:
    """LST-like segmented parabolic dish (Sec. 3): hexagonal spherical facets
    1.51 m flat-to-flat on the paraboloid z = rho^2 / 4f, f = 28 m, each with
    R = 2 |centre - focus| and its normal bisecting +z and the direction to the
    focus; four 0.2 m masts to a 3 x 3 x 2 m camera box; focal plane 3 x 3 m at
    z = 28 m facing the dish.  Facet tilt errors: Gaussian per axis."""
    f = LST_F
    focus = np.array([0.0, 0.0, f])
    rng = _rng(seed, 2)
    mat = lst_reflectivity()
    mat.sigma = roughness
    surfs: List[Surface] = []
    # focal plane first (lowest id among the camera parts)
    surfs.append(Surface("sag", "focal", "rect", origin=(0.0, 0.0, f), rot=FACING_DOWN, ap=(1.5, 1.5, 0, 0)))
    centres = lst_facet_centres(n_facets)
    tilts = rng.normal(0.0, 1.0, size=(len(centres), 2)) * tilt_sigma
    for (x, y), tl in zip(centres, tilts):
        c = np.array([x, y, (x * x + y * y) / (4.0 * f)])
        to_f = (focus - c) / np.linalg.norm(focus - c)
        nrm = np.array([0.0, 0.0, 1.0]) + to_f
        nrm /= np.linalg.norm(nrm)
        R = 2.0 * np.linalg.norm(c - focus)
        surfs.append(Surface("sag", "mirror", "hexagon", material=0, origin=tuple(c.tolist()),
                             rot=frame_from_axis(nrm), tilt=(float(tl[0]), float(tl[1])), curv=1.0 / R,
                             ap=(LST_PITCH / 2.0, 0, 0, 0)))
    if with_structure:
        zb = f + 0.001  # box bottom 1 mm above the focal plane (no coincident faces)
        surfs.append(Surface("box", "obscuration", origin=(0.0, 0.0, 0.5 * (zb + 30.0)),
                             prm=(1.5, 1.5, 0.5 * (30.0 - zb), 0, 0, 0, 0, 0)))
        for k in range(4):
            phi = math.radians(45.0 + 90.0 * k)
            a = np.array([11.5 * math.cos(phi), 11.5 * math.sin(phi), 11.5 ** 2 / (4.0 * f)])
            b = np.array([1.5 * math.copysign(1.0, math.cos(phi)), 1.5 * math.copysign(1.0, math.sin(phi)), zb])
            surfs.append(Surface("cylinder", "obscuration", origin=tuple(a.tolist()),
                                 rot=frame_from_axis(b - a), prm=(0.1, float(np.linalg.norm(b - a)), 0, 0, 0, 0, 0, 0)))
    return Scene("lst", surfs, [mat], [Medium()], length_scale=46.6, focal_length=f)


# Schwarzschild-Couder-like synthetic prescription (the paper prints none).
SC_R1 = 392.0 / 15.0
SC_R2 = 7.0


def _sag_base(R, r):
    return R - math.sqrt(R * R - r * r)


def sct_scene(seed: int = 0, asph_scale: float = 1e-3) -> Scene:
    """SC-like two-mirror system: concave primary (R = 392/15 m, annulus
    4.4-9.7 m, rings of 16 and 32 panels), concave secondary facing down at
    z = 8.4 m (R = 7 m, annulus 0.8-5.4 m, rings of 8 and 16 panels), both
    with even-asphere terms r^2..r^16 drawn at a 1e-3 relative sag scale; a
    spherical focal surface (R = 1 m) at z = 6.4 m and an obscuring disk over
    the secondary hole."""
    rng = _rng(seed, 2)
    mat = Material(lam=[300.0, 600.0], refl=[0.9, 0.9], sigma=0.0)
    surfs: List[Surface] = []
    surfs.append(Surface("sag", "focal", "circle", origin=(0.0, 0.0, 6.4), curv=1.0, ap=(0.45, 0, 0, 0)))
    surfs.append(Surface("sag", "obscuration", "circle", origin=(0.0, 0.0, 8.5), ap=(0.45, 0, 0, 0)))

    def coeffs(R, rmax):
        eps = rng.normal(0.0, 1.0, size=8)
        s = _sag_base(R, rmax)
        return tuple(float(eps[k - 1] * asph_scale * s / rmax ** (2 * k)) for k in range(1, 9))

    def panels(R, origin, rot, rmin, rmax, rings, asph):
        rmid = 0.5 * (rmin + rmax)
        bounds = [(rmin, rmid), (rmid, rmax)]
        for (r0, r1), npan in zip(bounds, rings):
            for p in range(npan):
                phi0 = 2 * math.pi * p / npan
                phi1 = 2 * math.pi * (p + 1) / npan
                surfs.append(Surface("sag", "mirror", "sector", material=0, origin=origin, rot=rot,
                                     curv=1.0 / R, asph=asph, ap=(r0, r1, phi0, phi1)))

    a1 = coeffs(SC_R1, 4.85)
    a2 = coeffs(SC_R2, 2.7)
    panels(SC_R1, (0.0, 0.0, 0.0), (1, 0, 0, 0, 1, 0, 0, 0, 1), 2.2, 4.85, (16, 32), a1)
    panels(SC_R2, (0.0, 0.0, 8.4), FACING_DOWN, 0.4, 2.7, (8, 16), a2)
    return Scene("sct", surfs, [mat], [Medium()], length_scale=17.3, focal_length=5.6)


# GCT-like dual-mirror small telescope (the paper prints no prescription): the SC-like system
# above scaled to an effective focal length of 2.283 m (primary 3.95 m, secondary 2.2 m across),
# primary split into 6 petals, monolithic secondary, its own seeded asphere terms.
GCT_F = 2.283
GCT_S = GCT_F / 5.6


def gct_scene(seed: int = 0, asph_scale: float = 1e-3) -> Scene:
    """GCT-like Schwarzschild-Couder system: the SC-like prescription scaled by
    s = 2.283 / 5.6 (concave primary R = s 392/15 m, annulus s (4.4-9.7) m in
    6 petals; concave secondary R = 7 s m facing down at z = 8.4 s, one
    annulus s (0.8-5.4) m); even-asphere terms r^2..r^16 at a 1e-3 relative
    sag scale (Philox stream 2 of `seed`); spherical focal surface R = s m at
    z = 6.4 s; an obscuring disk over the secondary hole.  Paraxial effective
    focal length 2.283 m."""
    s = GCT_S
    rng = _rng(seed + 7_000_003, 2)
    mat = Material(lam=[300.0, 600.0], refl=[0.88, 0.9], sigma=0.0)
    surfs: List[Surface] = []
    surfs.append(Surface("sag", "focal", "circle", origin=(0.0, 0.0, 6.4 * s), curv=1.0 / s, ap=(0.45 * s, 0, 0, 0)))
    surfs.append(Surface("sag", "obscuration", "circle", origin=(0.0, 0.0, 8.5 * s), ap=(0.45 * s, 0, 0, 0)))

    def coeffs(R, rmax):
        eps = rng.normal(0.0, 1.0, size=8)
        sb = _sag_base(R, rmax)
        return tuple(float(eps[k - 1] * asph_scale * sb / rmax ** (2 * k)) for k in range(1, 9))

    R1, R2 = SC_R1 * s, SC_R2 * s
    a1 = coeffs(R1, 4.85 * s)
    a2 = coeffs(R2, 2.7 * s)
    for p in range(6):
        phi0, phi1 = 2 * math.pi * p / 6, 2 * math.pi * (p + 1) / 6
        surfs.append(Surface("sag", "mirror", "sector", material=0, curv=1.0 / R1, asph=a1,
                             ap=(2.2 * s, 4.85 * s, phi0, phi1)))
    surfs.append(Surface("sag", "mirror", "annulus", material=0, origin=(0.0, 0.0, 8.4 * s), rot=FACING_DOWN,
                         curv=1.0 / R2, asph=a2, ap=(0.4 * s, 2.7 * s, 0, 0)))
    return Scene("gct", surfs, [mat], [Medium()], length_scale=17.3 * s, focal_length=GCT_F)


# Hexagonal light concentrator (entrance 50 mm flat-to-flat, exit 25 mm).
CONE_A_IN = 0.025
CONE_A_OUT = 0.0125
CONE_WINDOW = 0.002
# PMMA, one-term Sellmeier fit of Sultanova et al., Acta Phys. Pol. A 116 (2009):
# n^2 - 1 = 1.1819 l^2 / (l^2 - 0.011313), l in micrometres.
PMMA = Medium(n_const=0.0, B=(1.1819, 0.0, 0.0), C=(0.011313, 0.0, 0.0))


def winston_profile(a_out=CONE_A_OUT, theta_max=math.radians(30.0)):
    """Control points (r, z) of the quadratic Bezier that is exactly the 2D
    compound-parabolic-concentrator wall: the parabola with focus at the
    opposite exit edge (-a_out, 0), axis tilted by theta_max, focal length
    a_out (1 + sin theta_max), from the exit edge to the entrance edge
    a_in = a_out / sin theta_max.  A parabola arc is a quadratic Bezier whose
    middle control point is the intersection of its end tangents."""
    st, ct = math.sin(theta_max), math.cos(theta_max)
    fp = a_out * (1.0 + st)
    F = np.array([-a_out, 0.0])
    up = np.array([-st, ct])      # vertex -> focus
    perp = np.array([ct, st])
    V = F - fp * up

    def P(X):
        return V + X * perp + (X * X / (4.0 * fp)) * up

    def dP(X):
        return perp + (X / (2.0 * fp)) * up

    a_in = a_out / st
    X0 = 2.0 * a_out * ct
    # the entrance edge: r-coordinate of P(X) equals a_in, the larger root
    # P_r(X) = V_r + X ct - st X^2 / (4 fp)
    qa, qb, qc = -st / (4.0 * fp), ct, V[0] - a_in
    disc = qb * qb - 4 * qa * qc
    roots = [(-qb + math.sqrt(disc)) / (2 * qa), (-qb - math.sqrt(disc)) / (2 * qa)]
    X1 = min(r for r in roots if r > X0)
    P0, P2 = P(X0), P(X1)
    P1 = P0 + 0.5 * (X1 - X0) * dP(X0)
    return (float(P0[0]), float(P0[1])), (float(P1[0]), float(P1[1])), (float(P2[0]), float(P2[1]))


def cone_surfaces(H: float, p1: Sequence[float], window: bool = True, refl: float = 0.9,
                  mat_index: int = 0) -> List[Surface]:
    """Exit plane (focal role) at z = 0, Bezier hexagonal cone from apothem
    12.5 mm at z = 0 to 25 mm at z = H, optional 2 mm PMMA window on top with
    obscuring side faces."""
    s: List[Surface] = []
    s.append(Surface("sag", "focal", "hexagon", ap=(CONE_A_OUT, 0, 0, 0)))
    s.append(Surface("hexcone", "mirror", material=mat_index,
                     prm=(CONE_A_OUT, 0.0, p1[0], p1[1], CONE_A_IN, H, 0, 0)))
    if window:
        s.append(Surface("sag", "refract", "hexagon", origin=(0.0, 0.0, H), medium_front=1, medium_back=0,
                         ap=(CONE_A_IN, 0, 0, 0)))
        s.append(Surface("sag", "refract", "hexagon", origin=(0.0, 0.0, H + CONE_WINDOW), medium_front=0,
                         medium_back=1, ap=(CONE_A_IN, 0, 0, 0)))
        s.append(Surface("hexcone", "obscuration",
                         prm=(CONE_A_IN, H, CONE_A_IN, H + 0.5 * CONE_WINDOW, CONE_A_IN, H + CONE_WINDOW, 0, 0)))
    return s


def cone_variant_p1(v: int, n_variants: int = 64, seed: int = 0, jitter: float = 0.1):
    """Height and middle control point of variant v: H = 45 + 25 v / (n-1) mm;
    P1 = the Winston control point with z scaled to H, each coordinate
    jittered uniformly by +-10%."""
    H = 0.045 + 0.025 * (v / max(n_variants - 1, 1))
    P0, P1, P2 = winston_profile()
    rng = _rng(seed * 1000003 + v, 2)
    j = 1.0 + jitter * (2.0 * rng.random(2) - 1.0)
    p1 = (P1[0] * j[0], P1[1] * (H / P2[1]) * j[1])
    return H, p1


def cone_scene(n_variants: int = 1, seed: int = 0, window: bool = True, refl: float = 0.9) -> Scene:
    surfs: List[Surface] = []
    offs = [0]
    for v in range(n_variants):
        H, p1 = cone_variant_p1(v, n_variants, seed)
        surfs += cone_surfaces(H, p1, window=window, refl=refl)
        offs.append(len(surfs))
    mats = [Material(lam=[300.0], refl=[refl], sigma=0.0)]
    return Scene("cone", surfs, mats, [Medium(), PMMA], length_scale=0.1, focal_length=0.05,
                 variant_offsets=offs if n_variants > 1 else None)


def cone_heights(n_variants: int = 64, seed: int = 0):
    return [cone_variant_p1(v, n_variants, seed)[0] for v in range(n_variants)]


# ------------------------------------------------------------------ bundles
@dataclasses.dataclass
class Bundle:
    origins: np.ndarray      # [3, n] float64
    dirs: np.ndarray         # [3, n] float64
    wavelengths: np.ndarray  # [n] float64, nm

    @property
    def n(self):
        return self.wavelengths.shape[0]

    def astype(self, dtype):
        return Bundle(self.origins.astype(dtype), self.dirs.astype(dtype), self.wavelengths.astype(dtype))

    def rounded_to(self, dtype):
        """The bundle rounded to `dtype` and promoted back to float64."""
        return Bundle(self.origins.astype(dtype).astype(np.float64), self.dirs.astype(dtype).astype(np.float64),
                      self.wavelengths.astype(dtype).astype(np.float64))


def disk_bundle(n: int, radius: float, z_top: float, theta: float = 0.0, lam=(400.0, 400.0), seed: int = 0,
                stream: int = 1) -> Bundle:
    """Parallel bundle: direction d = (0, sin theta, -cos theta); origins
    uniform over a disk of `radius` perpendicular to d, centred where the line
    through the origin along d crosses z = z_top."""
    rng = _rng(seed, stream)
    u1 = rng.random(n)
    u2 = rng.random(n)
    d = np.array([0.0, math.sin(theta), -math.cos(theta)])
    centre = -d * (z_top / math.cos(theta))
    e1 = np.array([1.0, 0.0, 0.0])
    e2 = np.cross(d, e1)
    r = radius * np.sqrt(u1)
    ang = 2.0 * math.pi * u2
    o = centre[:, None] + r * (np.cos(ang) * e1[:, None] + np.sin(ang) * e2[:, None])
    dirs = np.repeat(d[:, None], n, axis=1)
    if lam[0] == lam[1]:
        wl = np.full(n, float(lam[0]))
    else:
        wl = lam[0] + (lam[1] - lam[0]) * rng.random(n)
    return Bundle(np.ascontiguousarray(o), np.ascontiguousarray(dirs), wl)


def hexagon_bundle(n: int, apothem: float, z0: float, theta: float, lam=(300.0, 600.0), seed: int = 0,
                   stream: int = 1) -> Bundle:
    """Origins uniform over the hexagon (flats at 0, 60, 120 deg) at height z0,
    direction tilted by theta towards the flat at azimuth 0:
    d = (sin theta, 0, -cos theta)."""
    rng = _rng(seed, stream)
    pts = np.empty((0, 2))
    R = apothem * 2.0 / math.sqrt(3.0)
    while pts.shape[0] < n:
        m = int((n - pts.shape[0]) * 1.3) + 16
        xy = (2.0 * rng.random((m, 2)) - 1.0) * np.array([apothem, R])
        x, y = xy[:, 0], xy[:, 1]
        inside = np.maximum.reduce([np.abs(x), np.abs(0.5 * x + math.sqrt(3) / 2 * y),
                                    np.abs(-0.5 * x + math.sqrt(3) / 2 * y)]) <= apothem
        pts = np.concatenate([pts, xy[inside]])
    pts = pts[:n]
    o = np.stack([pts[:, 0], pts[:, 1], np.full(n, z0)])
    d = np.array([math.sin(theta), 0.0, -math.cos(theta)])
    dirs = np.repeat(d[:, None], n, axis=1)
    wl = lam[0] + (lam[1] - lam[0]) * rng.random(n) if lam[0] != lam[1] else np.full(n, float(lam[0]))
    return Bundle(np.ascontiguousarray(o), np.ascontiguousarray(dirs), wl)


def concat(bundles: Sequence[Bundle]) -> Bundle:
    return Bundle(np.concatenate([b.origins for b in bundles], axis=1),
                  np.concatenate([b.dirs for b in bundles], axis=1),
                  np.concatenate([b.wavelengths for b in bundles]))


# ------------------------------------------------------- standard workloads
def sphere_workload(n: int = 100_000, seed: int = 0):
    """Single spherical mirror, 1e5 photons on a 1.2 m disk at z = 6 m, on axis, 400 nm."""
    return sphere_scene(), disk_bundle(n, 0.6, 6.0, 0.0, (400.0, 400.0), seed)


LST_ANGLES_DEG = (0.0, 0.5, 1.0, 1.5, 2.0)


def lst_workload(n_per_angle: int, seed: int = 0, angles_deg=LST_ANGLES_DEG):
    """LST-like dish: n photons per field angle on a 12 m disk from z = 32 m,
    wavelength uniform over 300-600 nm."""
    scene = lst_scene(seed=seed)
    bs = [disk_bundle(n_per_angle, 12.0, 32.0, math.radians(a), (300.0, 600.0), seed, stream=100 + k)
          for k, a in enumerate(angles_deg)]
    return scene, concat(bs)


SCT_ANGLES_DEG = tuple(4.0 * k / 7.0 for k in range(8))


def sct_workload(n_per_angle: int, seed: int = 0, angles_deg=SCT_ANGLES_DEG):
    scene = sct_scene(seed=seed)
    bs = [disk_bundle(n_per_angle, 5.0, 10.0, math.radians(a), (300.0, 600.0), seed, stream=200 + k)
          for k, a in enumerate(angles_deg)]
    return scene, concat(bs)


GCT_ANGLES_DEG = (0.0, 1.0, 2.0, 3.0, 4.0)


def gct_workload(n_per_angle: int, seed: int = 0, angles_deg=GCT_ANGLES_DEG):
    """GCT-like system: n photons per field angle on a 2.1 m disk from z = 10 s,
    wavelength uniform over 300-600 nm."""
    scene = gct_scene(seed=seed)
    bs = [disk_bundle(n_per_angle, 5.0 * GCT_S, 10.0 * GCT_S, math.radians(a), (300.0, 600.0), seed, stream=250 + k)
          for k, a in enumerate(angles_deg)]
    return scene, concat(bs)


CONE_ANGLES_DEG = tuple(float(a) for a in range(41))


def cone_batch(n_variants: int = 64, angles_deg=CONE_ANGLES_DEG, n_per_group: int = 2_000_000, seed: int = 0,
               lam=(300.0, 600.0)):
    """Batched hexagonal-concentrator study: n_variants cone designs (one
    scene with variant offsets) and one source group per (variant, incidence
    angle): photons uniform over the 50 mm entrance hexagon, 0.1 mm above the
    window, tilted towards the flat at azimuth 0."""
    scene = cone_scene(n_variants=n_variants, seed=seed)
    Hs = cone_heights(n_variants, seed=seed)
    groups = []
    for v in range(n_variants):
        for a in angles_deg:
            th = math.radians(a)
            groups.append(dict(variant=v, n=int(n_per_group), centre=(0.0, 0.0, Hs[v] + CONE_WINDOW + 1e-4),
                               apothem=CONE_A_IN, dir=(math.sin(th), 0.0, -math.cos(th)), lam=lam,
                               angle_deg=a))
    return scene, groups


def dish_batch(n_dishes: int = 32, n_min: int = 60, n_max: int = 198, photons_per_dish: int = 1_000_000,
               angles_deg=None, seed: int = 0):
    """Differentiable batch: n_dishes LST-like dishes with facet counts evenly
    spaced over [n_min, n_max] (the first N lattice facets by radius), each
    with its own focal plane, masts and camera box, as the variants of one
    scene.  Photons: photons_per_dish per dish, split over angles_deg, or by
    default all at ONE field angle per dish, the angles spread evenly over
    0-2 deg across the dishes (so each dish's spot is one spot).
    Returns (scene, bundle, variant_of_photon, facet counts)."""
    surfs: List[Surface] = []
    offs = [0]
    bundles, vop = [], []
    counts = [int(round(n_min + (n_max - n_min) * v / max(n_dishes - 1, 1))) for v in range(n_dishes)]
    for v, nf in enumerate(counts):
        sc = lst_scene(seed=seed * 1000 + v, n_facets=nf)
        surfs += sc.surfaces
        offs.append(len(surfs))
        angles = angles_deg if angles_deg is not None else (2.0 * v / max(n_dishes - 1, 1),)
        per_angle = max(1, photons_per_dish // len(angles))
        for k, a in enumerate(angles):
            b = disk_bundle(per_angle, 12.0, 32.0, math.radians(a), (300.0, 600.0), seed * 1000 + v, stream=500 + k)
            bundles.append(b)
            vop.append(np.full(b.n, v, np.int32))
    scene = Scene("dish_batch", surfs, [lst_reflectivity()], [Medium()], length_scale=46.6, focal_length=LST_F,
                  variant_offsets=offs)
    return scene, concat(bundles), np.concatenate(vop), counts


def lens_scene(R1: float = 0.1, thickness: float = 0.01, aperture: float = 0.02, n: float = 1.49,
               abs_len=None, asph=(0.0,) * 8, focal_z=None) -> Scene:
    """A thick plano-convex lens (the refracting counterpart of the mirrors,
    Sec. 2.1 ALens): convex spherical (or even-aspheric) front of radius R1
    facing +z with its vertex at z = thickness, flat back face at z = 0,
    medium 1 of constant index n (optionally absorbing: abs_len = (lam list,
    length list)); optionally a focal plane facing +z at z = focal_z."""
    med = Medium(n_const=n)
    if abs_len is not None:
        med = Medium(n_const=n, abs_lam=tuple(abs_len[0]), abs_len=tuple(abs_len[1]))
    surfs = [Surface("sag", "refract", "circle", origin=(0.0, 0.0, thickness), curv=-1.0 / R1, asph=tuple(asph),
                     medium_front=0, medium_back=1, ap=(aperture, 0, 0, 0)),
             Surface("sag", "refract", "circle", origin=(0.0, 0.0, 0.0), medium_front=1, medium_back=0,
                     ap=(aperture, 0, 0, 0))]
    if focal_z is not None:
        surfs.append(Surface("sag", "focal", "circle", origin=(0.0, 0.0, focal_z), ap=(aperture, 0, 0, 0)))
    fl = R1 / (n - 1.0)
    return Scene("lens", surfs, [Material([400.0], [1.0])], [Medium(), med], length_scale=max(0.1, 2 * fl),
                 focal_length=fl)


def tolerance_sweep(n_realizations: int = 16, tilt_sigma: float = 0.5e-3, photons_per_realization: int = 100_000,
                    field_deg: float = 1.0, seed: int = 0, n_facets: Optional[int] = None):
    """Misalignment study (Sec. 3: tolerance analysis): n_realizations copies of
    the LST-like dish, each with its own Gaussian facet-tilt errors (sigma per
    axis), as the variants of one scene; the same photon bundle (one field
    angle) traced through each.  Returns (scene, bundle, variant_of_photon);
    photons of realization v are the contiguous range v*n .. (v+1)*n - 1."""
    surfs: List[Surface] = []
    offs = [0]
    for v in range(n_realizations):
        sc = lst_scene(tilt_sigma=tilt_sigma, seed=seed * 1000 + 17 * v + 1, n_facets=n_facets)
        surfs += sc.surfaces
        offs.append(len(surfs))
    b = disk_bundle(photons_per_realization, 12.0, 32.0, math.radians(field_deg), (300.0, 600.0), seed, stream=900)
    bundle = concat([b] * n_realizations)
    vop = np.repeat(np.arange(n_realizations, dtype=np.int32), b.n)
    scene = Scene("tolerance", surfs, [lst_reflectivity()], [Medium()], length_scale=46.6, focal_length=LST_F,
                  variant_offsets=offs)
    return scene, bundle, vop
