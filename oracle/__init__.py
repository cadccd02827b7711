"""FP64 CPU oracle for the non-sequential photon trace -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The CUDA library never does; the two
share no code.  The C++ source (`oracle.cpp`) is a plain brute-force scalar
tracer in double precision; this module compiles it with gcc and marshals the
plain-Python scene records of `workloads` into the oracle's own structs.

Every function of the tracer is pinned by tests against closed forms,
invariants, an independent library routine (libcurand's Philox) or brute force
(tests/test_oracle_*.py).  Parity unpinned: the absolute PSF R80, effective
area and collection efficiency of the synthetic dish, two-mirror and cone
systems (the paper prints no values); they are compared only GPU vs oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_SHAPES = {"sag": 0, "cylinder": 1, "box": 2, "hexcone": 3}
_ROLES = {"mirror": 0, "refract": 1, "focal": 2, "obscuration": 3}
_APS = {"none": 0, "circle": 1, "annulus": 2, "sector": 3, "hexagon": 4, "rect": 5}


class OSurface(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("role", ctypes.c_int32), ("aperture", ctypes.c_int32),
                ("material", ctypes.c_int32), ("medium_front", ctypes.c_int32), ("medium_back", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("origin", ctypes.c_double * 3), ("rot", ctypes.c_double * 9),
                ("tilt", ctypes.c_double * 2), ("curv", ctypes.c_double), ("conic", ctypes.c_double),
                ("asph", ctypes.c_double * 8), ("ap", ctypes.c_double * 4), ("prm", ctypes.c_double * 8)]


class OMaterial(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pad", ctypes.c_int32), ("lam", ctypes.c_double * 16),
                ("refl", ctypes.c_double * 16), ("sigma", ctypes.c_double)]


class OMedium(ctypes.Structure):
    _fields_ = [("n_const", ctypes.c_double), ("B", ctypes.c_double * 3), ("C", ctypes.c_double * 3),
                ("n_abs", ctypes.c_int32), ("pad", ctypes.c_int32), ("abs_lam", ctypes.c_double * 16),
                ("abs_len", ctypes.c_double * 16)]


class OScene(ctypes.Structure):
    _fields_ = [("n_surfaces", ctypes.c_int32), ("n_materials", ctypes.c_int32), ("n_media", ctypes.c_int32),
                ("n_variants", ctypes.c_int32), ("surfaces", ctypes.POINTER(OSurface)),
                ("materials", ctypes.POINTER(OMaterial)), ("media", ctypes.POINTER(OMedium)),
                ("variant_offsets", ctypes.POINTER(ctypes.c_int32))]


class OSourceGroup(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("pad", ctypes.c_int32), ("first", ctypes.c_int64),
                ("n", ctypes.c_int64), ("c", ctypes.c_double * 3), ("apothem", ctypes.c_double),
                ("dir", ctypes.c_double * 3), ("lam_min", ctypes.c_double), ("lam_max", ctypes.c_double)]


class OOutputs(ctypes.Structure):
    _fields_ = [("status", ctypes.c_void_p), ("bounces", ctypes.c_void_p), ("hit", ctypes.c_void_p),
                ("dir", ctypes.c_void_p), ("last_surface", ctypes.c_void_p), ("focal_xy", ctypes.c_void_p),
                ("edge_margin", ctypes.c_void_p), ("cond", ctypes.c_void_p)]


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.oracle_trace.restype = ctypes.c_int
            _lib.oracle_trace.argtypes = [ctypes.POINTER(OScene), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                          ctypes.POINTER(OOutputs)]
            _lib.oracle_fresnel_unpolarised.restype = ctypes.c_double
            _lib.oracle_fresnel_unpolarised.argtypes = [ctypes.c_double] * 3
            _lib.oracle_refractive_index.restype = ctypes.c_double
            _lib.oracle_refractive_index.argtypes = [ctypes.POINTER(OMedium), ctypes.c_double]
            _lib.oracle_absorption_length.restype = ctypes.c_double
            _lib.oracle_absorption_length.argtypes = [ctypes.POINTER(OMedium), ctypes.c_double]
            _lib.oracle_reflectivity.restype = ctypes.c_double
            _lib.oracle_reflectivity.argtypes = [ctypes.POINTER(OMaterial), ctypes.c_double]
            _lib.oracle_philox4x32_10.restype = None
            _lib.oracle_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_generate_sources.restype = ctypes.c_int64
            _lib.oracle_generate_sources.argtypes = [ctypes.POINTER(OSourceGroup), ctypes.c_int32, ctypes.c_uint64,
                                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_objective.restype = ctypes.c_int
            _lib.oracle_objective.argtypes = [ctypes.POINTER(OScene), ctypes.c_int64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                              ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]
            _lib.oracle_track.restype = ctypes.c_int64
            _lib.oracle_track.argtypes = [ctypes.POINTER(OScene), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            _lib.oracle_intersect.restype = ctypes.c_int
            _lib.oracle_intersect.argtypes = [ctypes.POINTER(OSurface), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                              ctypes.c_void_p]
        return _lib


def _fill(arr, vals):
    for i, v in enumerate(vals):
        arr[i] = float(v)


def pack_surface(s) -> OSurface:
    o = OSurface()
    o.shape = _SHAPES[s.shape]
    o.role = _ROLES[s.role]
    o.aperture = _APS[s.aperture]
    o.material, o.medium_front, o.medium_back = int(s.material), int(s.medium_front), int(s.medium_back)
    _fill(o.origin, s.origin)
    _fill(o.rot, s.rot)
    _fill(o.tilt, s.tilt)
    o.curv, o.conic = float(s.curv), float(s.conic)
    _fill(o.asph, list(s.asph) + [0.0] * (8 - len(s.asph)))
    _fill(o.ap, list(s.ap) + [0.0] * (4 - len(s.ap)))
    _fill(o.prm, list(s.prm) + [0.0] * (8 - len(s.prm)))
    return o


def pack_material(m) -> OMaterial:
    o = OMaterial()
    o.n = len(m.lam)
    _fill(o.lam, m.lam)
    _fill(o.refl, m.refl)
    o.sigma = float(m.sigma)
    return o


def pack_medium(m) -> OMedium:
    o = OMedium()
    o.n_const = float(m.n_const)
    _fill(o.B, m.B)
    _fill(o.C, m.C)
    lam = list(getattr(m, "abs_lam", ()) or ())
    ln = list(getattr(m, "abs_len", ()) or ())
    o.n_abs = len(lam)
    _fill(o.abs_lam, lam)
    _fill(o.abs_len, ln)
    return o


class PackedScene:
    """Keeps the ctypes arrays alive while the oracle uses them."""

    def __init__(self, scene):
        self.surfs = (OSurface * len(scene.surfaces))(*[pack_surface(s) for s in scene.surfaces])
        self.mats = (OMaterial * max(1, len(scene.materials)))(*[pack_material(m) for m in scene.materials])
        self.meds = (OMedium * max(1, len(scene.media)))(*[pack_medium(m) for m in scene.media])
        self.offs = None
        self.s = OScene()
        self.s.n_surfaces = len(scene.surfaces)
        self.s.n_materials = len(scene.materials)
        self.s.n_media = len(scene.media)
        self.s.surfaces = self.surfs
        self.s.materials = self.mats
        self.s.media = self.meds
        if scene.variant_offsets is not None:
            self.offs = (ctypes.c_int32 * len(scene.variant_offsets))(*scene.variant_offsets)
            self.s.n_variants = len(scene.variant_offsets) - 1
            self.s.variant_offsets = self.offs
        else:
            self.s.n_variants = 1


def default_eps(scene, precision: int = 64) -> float:
    """Self-intersection epsilon: 1e-9 L_sys for the FP64 trace, 1e-6 L_sys for FP32."""
    return scene.length_scale * (1e-9 if precision == 64 else 1e-6)


def trace(scene, bundle, seed: int = 0, first_photon_id: int = 0, max_bounces: int = 100, eps=None,
          variant_of_photon=None, n_threads: int = 0, precision_eps: int = 64):
    """Trace a bundle with the oracle.  Returns a dict of numpy arrays."""
    L = lib()
    n = bundle.n
    o = np.ascontiguousarray(bundle.origins, dtype=np.float64).reshape(3, n)
    d = np.ascontiguousarray(bundle.dirs, dtype=np.float64).reshape(3, n)
    wl = np.ascontiguousarray(bundle.wavelengths, dtype=np.float64)
    if eps is None:
        eps = default_eps(scene, precision_eps)
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    res = {
        "status": np.zeros(n, np.uint8), "bounces": np.zeros(n, np.uint8), "hit": np.zeros((3, n)),
        "dir": np.zeros((3, n)), "last_surface": np.zeros(n, np.int32), "focal_xy": np.zeros((2, n)),
        "edge_margin": np.zeros(n), "cond": np.zeros(n),
    }
    outs = OOutputs(*[res[k].ctypes.data for k in
                      ("status", "bounces", "hit", "dir", "last_surface", "focal_xy", "edge_margin", "cond")])
    vop = None
    if variant_of_photon is not None:
        vop = np.ascontiguousarray(variant_of_photon, dtype=np.int32)
    ps = PackedScene(scene)
    rc = L.oracle_trace(ctypes.byref(ps.s), n, o.ctypes.data, d.ctypes.data, wl.ctypes.data,
                        vop.ctypes.data if vop is not None else None, seed & (2**64 - 1), first_photon_id,
                        max_bounces, float(eps), n_threads, ctypes.byref(outs))
    if rc != 0:
        raise ValueError(f"oracle_trace rejected the scene or arguments (code {rc})")
    return res


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def fresnel(n1, n2, cos_i):
    return lib().oracle_fresnel_unpolarised(n1, n2, cos_i)


def refractive_index(medium, lam_nm):
    m = pack_medium(medium)
    return lib().oracle_refractive_index(ctypes.byref(m), lam_nm)


def reflectivity(material, lam_nm):
    m = pack_material(material)
    return lib().oracle_reflectivity(ctypes.byref(m), lam_nm)


def intersect(surface, p, d, eps=1e-12):
    """Nearest hit of one ray with one surface: (t, front normal, local point) or None."""
    s = pack_surface(surface)
    pa = np.ascontiguousarray(p, np.float64)
    da = np.ascontiguousarray(d, np.float64)
    t = ctypes.c_double()
    nf = np.zeros(3)
    lp = np.zeros(3)
    rc = lib().oracle_intersect(ctypes.byref(s), pa.ctypes.data, da.ctypes.data, eps, ctypes.byref(t),
                                nf.ctypes.data, lp.ctypes.data)
    if rc < 0:
        raise ArithmeticError("Newton iteration did not converge")
    if rc == 0:
        return None
    return t.value, nf, lp


def generate_sources(groups, seed: int = 0, first_photon_id: int = 0):
    """Photons of source groups from Philox stream 1 (see oracle_generate_sources).

    groups: list of dicts with keys variant, n, centre (3), apothem, dir (3),
    lam (min, max); photons are numbered in group order.  Returns (Bundle-like
    dict with origins [3, n], dirs [3, n], wavelengths [n]), variant [n], and
    the number of photons with no accepted draw.
    """
    ng = len(groups)
    arr = (OSourceGroup * ng)()
    first = 0
    for k, g in enumerate(groups):
        a = arr[k]
        a.variant = int(g["variant"])
        a.first = first
        a.n = int(g["n"])
        _fill(a.c, g["centre"])
        a.apothem = float(g["apothem"])
        _fill(a.dir, g["dir"])
        a.lam_min, a.lam_max = float(g["lam"][0]), float(g["lam"][1])
        first += int(g["n"])
    n = first
    o = np.zeros((3, n))
    d = np.zeros((3, n))
    lam = np.zeros(n)
    var = np.zeros(n, np.int32)
    failed = lib().oracle_generate_sources(arr, ng, seed & (2**64 - 1), first_photon_id, o.ctypes.data,
                                           d.ctypes.data, lam.ctypes.data, var.ctypes.data)
    return {"origins": o, "dirs": d, "wavelengths": lam}, var, int(failed)


N_PARAM = 16
OBJECTIVES = {"msr": 0, "soft_ce": 1, "centroid_x": 2, "centroid_y": 3}


def objective(scene, bundle, objective="msr", seed=0, first_photon_id=0, max_bounces=100, eps=None,
              variant_of_photon=None, tau=0.5e-3, delta=None, grad=True, n_threads=0):
    """Frozen-path objective (and its gradient by dual numbers) -- see oracle.h.

    delta: optional [n_surfaces, 16] parameter offsets (tilt x, y; A1..A8;
    Bezier P0r, P0z, P1r, P1z, P2r, P2z).  Returns (value, grad [n_surfaces, 16] or None).
    """
    L = lib()
    n = bundle.n
    o = np.ascontiguousarray(bundle.origins, dtype=np.float64).reshape(3, n)
    d = np.ascontiguousarray(bundle.dirs, dtype=np.float64).reshape(3, n)
    wl = np.ascontiguousarray(bundle.wavelengths, dtype=np.float64)
    if eps is None:
        eps = default_eps(scene, 64)
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    ns = len(scene.surfaces)
    dl = None
    if delta is not None:
        dl = np.ascontiguousarray(delta, dtype=np.float64).reshape(ns, N_PARAM)
    g = np.zeros((ns, N_PARAM)) if grad else None
    vop = None if variant_of_photon is None else np.ascontiguousarray(variant_of_photon, dtype=np.int32)
    val = ctypes.c_double()
    ps = PackedScene(scene)
    rc = L.oracle_objective(ctypes.byref(ps.s), n, o.ctypes.data, d.ctypes.data, wl.ctypes.data,
                            vop.ctypes.data if vop is not None else None, seed & (2**64 - 1), first_photon_id,
                            max_bounces, float(eps), n_threads, OBJECTIVES[objective], float(tau),
                            dl.ctypes.data if dl is not None else None, ctypes.byref(val),
                            g.ctypes.data if g is not None else None)
    if rc != 0:
        raise ValueError(f"oracle_objective failed (code {rc})")
    return val.value, g


def track(scene, bundle, first, count, seed=0, first_photon_id=0, max_bounces=100, eps=None, variant_of_photon=None,
          cap=100_000):
    """Interaction records of photons first .. first+count-1: (points [k, 3], info [k, 4] =
    photon index, bounce, surface id, status after), photon then bounce order."""
    L = lib()
    n = bundle.n
    o = np.ascontiguousarray(bundle.origins, dtype=np.float64).reshape(3, n)
    d = np.ascontiguousarray(bundle.dirs, dtype=np.float64).reshape(3, n)
    wl = np.ascontiguousarray(bundle.wavelengths, dtype=np.float64)
    if eps is None:
        eps = default_eps(scene, 64)
    pts = np.zeros((cap, 3))
    info = np.zeros((cap, 4), np.int32)
    vop = None if variant_of_photon is None else np.ascontiguousarray(variant_of_photon, dtype=np.int32)
    ps = PackedScene(scene)
    k = L.oracle_track(ctypes.byref(ps.s), n, o.ctypes.data, d.ctypes.data, wl.ctypes.data,
                       vop.ctypes.data if vop is not None else None, seed & (2**64 - 1), first_photon_id,
                       max_bounces, float(eps), first, count, pts.ctypes.data, info.ctypes.data, cap)
    if k < 0:
        raise ValueError("oracle_track: bad arguments")
    k = min(int(k), cap)
    return pts[:k], info[:k]
