"""Python binding of the GB300 non-sequential photon tracer (include/robast.h).

Argument marshalling only: every step of the trace runs in the CUDA library
(`_build/librobast.so`, built from csrc/ for sm_103a).  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library cannot
be loaded, every call raises.

Typical use:

    import paper_1508_07803_gb300 as robast
    geom = robast.build_geometry(scene)          # scene: surfaces/materials/media records
    out = robast.trace(geom, origins, dirs, wavelengths, seed=0, precision=32)

`origins` and `dirs` are CUDA tensors of shape [3, n] (x row, y row, z row),
`wavelengths` [n] in nm; float32 for precision 32, float64 for precision 64.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

__all__ = ["build_geometry", "trace", "trace_host", "psf", "Geometry", "load", "STATUS", "RobastError"]

STATUS = {1: "DETECTED", 2: "ABSORBED", 3: "OBSCURED", 4: "ESCAPED", 5: "MAX_BOUNCES", 6: "ERROR"}
N_COUNTERS = 8

_SHAPES = {"sag": 0, "cylinder": 1, "box": 2, "hexcone": 3}
_ROLES = {"mirror": 0, "refract": 1, "focal": 2, "obscuration": 3}
_APS = {"none": 0, "circle": 1, "annulus": 2, "sector": 3, "hexagon": 4, "rect": 5}


class RobastError(RuntimeError):
    pass


class SurfaceDesc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("role", ctypes.c_int32), ("aperture", ctypes.c_int32),
                ("material", ctypes.c_int32), ("medium_front", ctypes.c_int32), ("medium_back", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("origin", ctypes.c_double * 3), ("rot", ctypes.c_double * 9),
                ("tilt", ctypes.c_double * 2), ("curv", ctypes.c_double), ("conic", ctypes.c_double),
                ("asph", ctypes.c_double * 8), ("ap", ctypes.c_double * 4), ("prm", ctypes.c_double * 8)]


class MaterialDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lam", ctypes.c_double * 16),
                ("refl", ctypes.c_double * 16), ("sigma", ctypes.c_double)]


class MediumDesc(ctypes.Structure):
    _fields_ = [("n_const", ctypes.c_double), ("B", ctypes.c_double * 3), ("C", ctypes.c_double * 3),
                ("n_abs", ctypes.c_int32), ("reserved", ctypes.c_int32), ("abs_lam", ctypes.c_double * 16),
                ("abs_len", ctypes.c_double * 16)]


class GeomDesc(ctypes.Structure):
    _fields_ = [("n_surfaces", ctypes.c_int32), ("n_materials", ctypes.c_int32), ("n_media", ctypes.c_int32),
                ("n_variants", ctypes.c_int32), ("surfaces", ctypes.POINTER(SurfaceDesc)),
                ("materials", ctypes.POINTER(MaterialDesc)), ("media", ctypes.POINTER(MediumDesc)),
                ("variant_offsets", ctypes.POINTER(ctypes.c_int32)), ("length_scale", ctypes.c_double)]


class TraceOut(ctypes.Structure):
    _fields_ = [("status", ctypes.c_void_p), ("bounces", ctypes.c_void_p), ("hit", ctypes.c_void_p),
                ("dir", ctypes.c_void_p), ("last_surface", ctypes.c_void_p), ("focal_xy", ctypes.c_void_p),
                ("counters", ctypes.c_void_p), ("err", ctypes.c_void_p), ("retraced", ctypes.c_void_p)]

OUT_FIELDS = ("status", "bounces", "hit", "dir", "last_surface", "focal_xy", "counters", "err", "retraced")


class TrackOpts(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("count", ctypes.c_int64), ("cap", ctypes.c_int64),
                ("points", ctypes.c_void_p), ("info", ctypes.c_void_p), ("n_records", ctypes.c_void_p)]


class TraceOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_bounces", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("variant_of_photon", ctypes.c_void_p), ("first_photon_id", ctypes.c_int64),
                ("eps", ctypes.c_double), ("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("work_units", ctypes.c_void_p), ("coherent_order", ctypes.c_int32),
                ("track", ctypes.POINTER(TrackOpts)), ("refill_min", ctypes.c_int32),
                ("accuracy_pos", ctypes.c_double), ("accuracy_dir", ctypes.c_double)]

# Default FP32 accuracy: final positions within 1e-6 of the system focal length, final
# directions within 1e-5 rad of an exact trace of the same inputs (the accuracy guard re-traces
# in FP64 every photon whose running error estimate exceeds 0.9 of either bound).
ACCURACY_REL_POS = 1e-6
ACCURACY_DIR = 1e-5

N_UNITS = 13
UNIT_NAMES = ("aabb", "sag", "newton", "aperture", "cylinder", "box", "hexwall", "reflect", "refract", "rough",
              "philox", "rebase", "refine")


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load librobast.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RobastError(f"CUDA library not built: {path} is missing (run paper_1508_07803_gb300.build.build())")
        lib = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.robast_build_geometry.argtypes = [ctypes.POINTER(GeomDesc), ctypes.POINTER(vp)]
        lib.robast_build_geometry.restype = ctypes.c_int
        lib.robast_free_geometry.argtypes = [vp]
        lib.robast_free_geometry.restype = None
        lib.robast_geometry_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.robast_trace.argtypes = [vp, vp, vp, vp, i64, ctypes.c_uint64, ctypes.POINTER(TraceOut)]
        lib.robast_trace_ex.argtypes = [vp, vp, vp, vp, i64, ctypes.c_uint64, ctypes.POINTER(TraceOut),
                                        ctypes.POINTER(TraceOpts)]
        lib.robast_trace_host.argtypes = [vp, vp, vp, vp, i64, ctypes.c_uint64, ctypes.POINTER(TraceOut),
                                          ctypes.POINTER(TraceOpts)]
        lib.robast_trace_opts_default.argtypes = [ctypes.POINTER(TraceOpts)]
        lib.robast_trace_opts_default.restype = None
        lib.robast_psf.argtypes = [vp, vp, vp, i64, i32, vp, vp, i32, vp, ctypes.POINTER(ctypes.c_double)]
        lib.robast_last_error.restype = ctypes.c_char_p
        lib.robast_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = _lib.robast_last_error().decode()
        raise RobastError(f"robast error {rc}: {msg}")


def _fill(arr, vals, n):
    vals = list(vals) + [0.0] * (n - len(vals))
    for i in range(n):
        arr[i] = float(vals[i])


def _pack(scene):
    surfs = (SurfaceDesc * len(scene.surfaces))()
    for k, s in enumerate(scene.surfaces):
        d = surfs[k]
        d.shape, d.role, d.aperture = _SHAPES[s.shape], _ROLES[s.role], _APS[s.aperture]
        d.material, d.medium_front, d.medium_back = int(s.material), int(s.medium_front), int(s.medium_back)
        _fill(d.origin, s.origin, 3)
        _fill(d.rot, s.rot, 9)
        _fill(d.tilt, s.tilt, 2)
        d.curv, d.conic = float(s.curv), float(s.conic)
        _fill(d.asph, s.asph, 8)
        _fill(d.ap, s.ap, 4)
        _fill(d.prm, s.prm, 8)
    mats = (MaterialDesc * max(1, len(scene.materials)))()
    for k, m in enumerate(scene.materials):
        mats[k].n = len(m.lam)
        _fill(mats[k].lam, m.lam, 16)
        _fill(mats[k].refl, m.refl, 16)
        mats[k].sigma = float(m.sigma)
    meds = (MediumDesc * max(1, len(scene.media)))()
    for k, m in enumerate(scene.media):
        meds[k].n_const = float(m.n_const)
        _fill(meds[k].B, m.B, 3)
        _fill(meds[k].C, m.C, 3)
        lam = list(getattr(m, "abs_lam", ()) or ())
        meds[k].n_abs = len(lam)
        _fill(meds[k].abs_lam, lam, 16)
        _fill(meds[k].abs_len, list(getattr(m, "abs_len", ()) or ()), 16)
    desc = GeomDesc()
    desc.n_surfaces = len(scene.surfaces)
    desc.n_materials = len(scene.materials)
    desc.n_media = len(scene.media)
    desc.surfaces = surfs
    desc.materials = mats
    desc.media = meds
    offs = None
    if getattr(scene, "variant_offsets", None) is not None:
        offs = (ctypes.c_int32 * len(scene.variant_offsets))(*scene.variant_offsets)
        desc.n_variants = len(scene.variant_offsets) - 1
        desc.variant_offsets = offs
    else:
        desc.n_variants = 1
    desc.length_scale = float(scene.length_scale)
    return desc, (surfs, mats, meds, offs)


class Geometry:
    """Device-resident optical system(s); frees its device tables on close/GC."""

    def __init__(self, handle, scene):
        self._h = ctypes.c_void_p(handle)
        self.length_scale = float(scene.length_scale)
        self.focal_length = float(scene.focal_length)
        self.n_surfaces = len(scene.surfaces)
        ns, nv, nn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.robast_geometry_info(self._h, ctypes.byref(ns), ctypes.byref(nv), ctypes.byref(nn)))
        self.n_variants, self.n_bvh_nodes = nv.value, nn.value

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RobastError("geometry already freed")
        return self._h

    def close(self):
        if self._h is not None and self._h.value and _lib is not None:
            _lib.robast_free_geometry(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_geometry(scene) -> Geometry:
    """robast_build_geometry: compile `scene` (surface/material/medium records) onto the current CUDA device."""
    lib = load()
    desc, keep = _pack(scene)
    h = ctypes.c_void_p()
    _check(lib.robast_build_geometry(ctypes.byref(desc), ctypes.byref(h)))
    del keep
    return Geometry(h.value, scene)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _trace_out(out):
    return TraceOut(*[(out[k].data_ptr() if out.get(k) is not None else None) for k in OUT_FIELDS])


def _accuracy(geom, precision, accuracy):
    """(position bound m, direction bound rad) of the FP32 accuracy guard: None = the default
    (1e-6 f, 1e-5 rad), False / 0 = off, or a pair."""
    if precision != 32 or accuracy is False or accuracy == 0:
        return 0.0, 0.0
    if accuracy is None:
        return ACCURACY_REL_POS * geom.focal_length, ACCURACY_DIR
    pos, ang = accuracy
    return float(pos or 0.0), float(ang or 0.0)


def _opts(precision, max_bounces, stream, vop_ptr, first_photon_id, eps, block_size, blocks_per_sm, units=None,
          coherent_order=0, refill_min=0, accuracy=(0.0, 0.0)):
    o = TraceOpts()
    _lib.robast_trace_opts_default(ctypes.byref(o))
    o.precision = int(precision)
    o.max_bounces = int(max_bounces)
    o.stream = stream
    o.variant_of_photon = vop_ptr
    o.first_photon_id = int(first_photon_id)
    o.eps = float(eps or 0.0)
    o.block_size = int(block_size)
    o.blocks_per_sm = int(blocks_per_sm)
    o.work_units = ctypes.c_void_p(units.data_ptr()) if units is not None else None
    o.coherent_order = int(coherent_order)
    o.refill_min = int(refill_min)
    o.accuracy_pos, o.accuracy_dir = float(accuracy[0]), float(accuracy[1])
    return o


def alloc_outputs(n: int, precision: int = 32, device="cuda", fields=None):
    """Output tensors for robast_trace (all fields unless `fields` restricts them)."""
    import torch
    dt = torch.float32 if precision == 32 else torch.float64
    all_fields = {
        "status": lambda: torch.empty(n, dtype=torch.uint8, device=device),
        "bounces": lambda: torch.empty(n, dtype=torch.uint8, device=device),
        "hit": lambda: torch.empty((3, n), dtype=dt, device=device),
        "dir": lambda: torch.empty((3, n), dtype=dt, device=device),
        "last_surface": lambda: torch.empty(n, dtype=torch.int32, device=device),
        "focal_xy": lambda: torch.empty((2, n), dtype=dt, device=device),
        "counters": lambda: torch.zeros(N_COUNTERS, dtype=torch.int64, device=device),
        "retraced": lambda: torch.zeros(2, dtype=torch.int64, device=device),
        "err": lambda: torch.empty((2, n), dtype=torch.float32, device=device),
    }
    keys = fields if fields is not None else [k for k in all_fields if k != "err" and (k != "retraced" or precision == 32)]
    return {k: all_fields[k]() for k in keys}


def trace(geom: Geometry, origins, dirs, wavelengths, seed: int = 0, precision: int = 32, max_bounces: int = 100,
          stream=None, variant_of_photon=None, first_photon_id: int = 0, eps: Optional[float] = None,
          block_size: int = 0, blocks_per_sm: int = 0, out: Optional[dict] = None, work_units=None,
          coherent_order: int = 0, track=None, refill_min: int = 0, accuracy=None, error_estimate: bool = False):
    """robast_trace_ex on CUDA tensors; returns the dict of output tensors.

    work_units: optional CUDA int64 tensor [N_UNITS]; when given, the counting
    build of the kernel runs and adds its work units (UNIT_NAMES) to it.
    block_size (64, 128, 256, or 512 for FP32), blocks_per_sm, coherent_order
    and refill_min (0..32: idle lanes a warp waits for before it takes new
    photons) shape the launch only: the results do not depend on them.
    accuracy (FP32): None = final positions within 1e-6 of the geometry's focal
    length and directions within 1e-5 rad of an exact trace, enforced by
    re-tracing in FP64 the photons whose running error estimate exceeds 0.9 of
    a bound; a (pos_m, dir_rad) pair sets the bounds; False turns the guard off.
    out["retraced"] counts (re-traced, over a bound but not re-traced).
    error_estimate: also return out["err"] [2, n] float32, the per-photon
    position / direction error estimate (-1 where the photon was re-traced).
    """
    import torch
    lib = load()
    dt = torch.float32 if precision == 32 else torch.float64
    n = int(wavelengths.shape[0])
    for name, t, shape in (("origins", origins, (3, n)), ("dirs", dirs, (3, n)), ("wavelengths", wavelengths, (n,))):
        if t.dtype != dt or tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous():
            raise RobastError(f"{name}: need a contiguous CUDA {dt} tensor of shape {shape}")
    if out is None:
        out = alloc_outputs(n, precision, origins.device)
        if error_estimate and precision == 32:
            out["err"] = torch.empty((2, n), dtype=torch.float32, device=origins.device)
    tout = _trace_out(out)
    if stream is None:
        stream = torch.cuda.current_stream(origins.device)
    sp = ctypes.c_void_p(stream.cuda_stream)
    vop = None
    if variant_of_photon is not None:
        if variant_of_photon.dtype != torch.int32 or not variant_of_photon.is_cuda:
            raise RobastError("variant_of_photon: need a CUDA int32 tensor")
        vop = ctypes.c_void_p(variant_of_photon.data_ptr())
    o = _opts(precision, max_bounces, sp, vop, first_photon_id, eps, block_size, blocks_per_sm, work_units,
              coherent_order, refill_min, _accuracy(geom, precision, accuracy))
    tr = None
    if track is not None:
        tr = TrackOpts(int(track["first"]), int(track["count"]), int(track["cap"]), track["points"].data_ptr(),
                       track["info"].data_ptr(), track["n_records"].data_ptr())
        o.track = ctypes.pointer(tr)
    _check(lib.robast_trace_ex(geom.handle, _ptr(origins), _ptr(dirs), _ptr(wavelengths), n,
                               ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(tout), ctypes.byref(o)))
    return out


def trace_host(geom: Geometry, origins, dirs, wavelengths, seed: int = 0, precision: int = 32,
               max_bounces: int = 100, stream=None, out: Optional[dict] = None, first_photon_id: int = 0,
               eps: Optional[float] = None, variant_of_photon=None, accuracy=None, error_estimate: bool = False):
    """robast_trace_host: host (CPU, ideally pinned) tensors in and out; synchronous.

    The photons go to the GPU in chunks over two streams, so copies overlap the
    trace; the results equal one robast.trace over all photons.  accuracy and
    error_estimate as for trace().
    """
    import torch
    lib = load()
    dt = torch.float32 if precision == 32 else torch.float64
    n = int(wavelengths.shape[0])
    for name, t in (("origins", origins), ("dirs", dirs), ("wavelengths", wavelengths)):
        if t.dtype != dt or t.is_cuda or not t.is_contiguous():
            raise RobastError(f"{name}: need a contiguous host {dt} tensor")
    if out is None:
        out = alloc_outputs(n, precision, "cpu")
        if error_estimate and precision == 32:
            out["err"] = torch.empty((2, n), dtype=torch.float32)
    tout = _trace_out(out)
    if stream is None:
        stream = torch.cuda.current_stream()
    vop = ctypes.c_void_p(variant_of_photon.data_ptr()) if variant_of_photon is not None else None
    o = _opts(precision, max_bounces, ctypes.c_void_p(stream.cuda_stream), vop, first_photon_id, eps, 0, 0,
              accuracy=_accuracy(geom, precision, accuracy))
    _check(lib.robast_trace_host(geom.handle, _ptr(origins), _ptr(dirs), _ptr(wavelengths), n,
                                 ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(tout), ctypes.byref(o)))
    return out


def psf(geom: Geometry, status, focal_xy, precision: int = 32, stream=None, start: int = 0, count=None,
        windows=None):
    """robast_psf: spot-diagram statistics (N_detected, cx, cy, R80) of DETECTED photons.

    status [N] and focal_xy [2, N] are trace outputs.  Either one window
    (start, count) -> one tuple, or `windows` = [(start, count), ...] -> a
    list of tuples, all reduced in one pass.
    """
    import torch
    lib = load()
    N = int(status.shape[0])
    single = windows is None
    if single:
        windows = [(start, N - start if count is None else int(count))]
    _check_spot_args(status, focal_xy, precision, "psf")
    if stream is None:
        stream = torch.cuda.current_stream(status.device)
    nw = len(windows)
    st = (ctypes.c_int64 * nw)(*[int(w[0]) for w in windows])
    ct = (ctypes.c_int64 * nw)(*[int(w[1]) for w in windows])
    res = (ctypes.c_double * (4 * nw))()
    with torch.cuda.device(status.device):
        _check(lib.robast_psf(geom.handle, _ptr(status), _ptr(focal_xy), N, nw, st, ct, int(precision),
                              ctypes.c_void_p(stream.cuda_stream), res))
    out = [tuple(res[4 * w:4 * w + 4]) for w in range(nw)]
    return out[0] if single else out


def _check_spot_args(status, focal_xy, precision, name):
    """The spot-diagram reductions read N status bytes and 2N focal coordinates of the
    precision's type from one device: anything else would read past the buffers."""
    import torch
    want = {32: torch.float32, 64: torch.float64}.get(int(precision))
    if want is None:
        raise RobastError(f"{name}: precision must be 32 or 64")
    N = int(status.shape[0]) if status.dim() == 1 else -1
    if status.dtype != torch.uint8 or status.dim() != 1 or not status.is_contiguous():
        raise RobastError(f"{name}: status must be a contiguous uint8 tensor [N]")
    if focal_xy.dtype != want or tuple(focal_xy.shape) != (2, N) or not focal_xy.is_contiguous():
        raise RobastError(f"{name}: focal_xy must be a contiguous {want} tensor [2, {N}] for precision {precision}")
    if not (status.is_cuda and focal_xy.is_cuda) or status.device != focal_xy.device:
        raise RobastError(f"{name}: status and focal_xy must be CUDA tensors on one device")


def version() -> str:
    return load().robast_version().decode()


def measure_alu_peak(precision: int = 32, stream=None) -> float:
    """robast_measure_alu_peak: FMA throughput of the current GPU in FLOP/s (roofline denominator)."""
    import torch
    lib = load()
    lib.robast_measure_alu_peak.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    if stream is None:
        stream = torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(lib.robast_measure_alu_peak(int(precision), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(v)))
    return v.value


def psf_noalloc(status, focal_xy, windows, precision: int = 32, stream=None):
    """robast_psf_noalloc: spot-diagram statistics per window without any allocation.

    For callers that cannot allocate device memory at this point; scratch is a
    fixed array inside the library (at most 64 windows per call).  Returns a
    list of (N_detected, cx, cy, R80) per window, like psf(..., windows=...).
    """
    import torch
    lib = load()
    lib.robast_psf_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double)]
    N = int(status.shape[0])
    _check_spot_args(status, focal_xy, precision, "psf_noalloc")
    if stream is None:
        stream = torch.cuda.current_stream(status.device)
    nw = len(windows)
    st = (ctypes.c_int64 * nw)(*[int(w[0]) for w in windows])
    ct = (ctypes.c_int64 * nw)(*[int(w[1]) for w in windows])
    res = (ctypes.c_double * (4 * nw))()
    with torch.cuda.device(status.device):
        _check(lib.robast_psf_noalloc(_ptr(status), _ptr(focal_xy), N, nw, st, ct, int(precision),
                                      ctypes.c_void_p(stream.cuda_stream), res))
    return [tuple(res[4 * w:4 * w + 4]) for w in range(nw)]


class SourceGroupDesc(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_photons", ctypes.c_int64),
                ("centre", ctypes.c_double * 3), ("apothem", ctypes.c_double), ("dir", ctypes.c_double * 3),
                ("lam_min", ctypes.c_double), ("lam_max", ctypes.c_double)]


class Sources:
    """Device-resident source groups (robast_sources_create)."""

    def __init__(self, handle, n_groups, n_photons):
        self._h = ctypes.c_void_p(handle)
        self.n_groups, self.n_photons = n_groups, n_photons

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RobastError("sources already freed")
        return self._h

    def close(self):
        if self._h is not None and self._h.value and _lib is not None:
            _lib.robast_sources_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sources_create(geom: Geometry, groups) -> Sources:
    """robast_sources_create from a list of dicts: variant, n, centre (3), apothem, dir (3), lam (min, max)."""
    lib = load()
    lib.robast_sources_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_void_p)]
    lib.robast_sources_free.argtypes = [ctypes.c_void_p]
    lib.robast_sources_free.restype = None
    lib.robast_sources_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]
    arr = (SourceGroupDesc * len(groups))()
    for k, g in enumerate(groups):
        a = arr[k]
        a.variant = int(g["variant"])
        a.n_photons = int(g["n"])
        _fill(a.centre, g["centre"], 3)
        a.apothem = float(g["apothem"])
        _fill(a.dir, g["dir"], 3)
        a.lam_min, a.lam_max = float(g["lam"][0]), float(g["lam"][1])
    h = ctypes.c_void_p()
    _check(lib.robast_sources_create(geom.handle, arr, len(groups), ctypes.byref(h)))
    ng, npho = ctypes.c_int32(), ctypes.c_int64()
    _check(lib.robast_sources_info(h, ctypes.byref(ng), ctypes.byref(npho)))
    return Sources(h.value, ng.value, npho.value)


def trace_sources(geom: Geometry, src: Sources, group_counts, seed: int = 0, precision: int = 32,
                  max_bounces: int = 100, stream=None, out: Optional[dict] = None, first_photon_id: int = 0,
                  eps: Optional[float] = None, block_size: int = 0, blocks_per_sm: int = 0, refill_min: int = 0,
                  accuracy=None, work_units=None, coherent_order: int = 0):
    """robast_trace_sources: trace every photon of the source groups in one launch.

    group_counts: CUDA int64 tensor [n_groups, 8], added to.  out: optional
    dict of per-photon output tensors (see alloc_outputs) for src.n_photons.
    accuracy as for trace() (FP32: the FP64 re-trace is a second launch).
    work_units: optional CUDA int64 tensor [N_UNITS] (FP32 only): run the
    counting build (block 128) and add its work units to it.
    coherent_order: -1 traces the photons in id order instead of sorting each
    chunk by the cell of its generated origins; the results are the same.
    """
    import torch
    lib = load()
    lib.robast_trace_sources.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.POINTER(TraceOut), ctypes.POINTER(TraceOpts)]
    if tuple(group_counts.shape) != (src.n_groups, N_COUNTERS) or group_counts.dtype != torch.int64 \
            or not group_counts.is_cuda:
        raise RobastError("trace_sources: group_counts must be a CUDA int64 tensor [n_groups, 8]")
    if stream is None:
        stream = torch.cuda.current_stream(group_counts.device)
    tout = None
    if out is not None:
        tout = _trace_out(out)
    o = _opts(precision, max_bounces, ctypes.c_void_p(stream.cuda_stream), None, first_photon_id, eps, block_size,
              blocks_per_sm, units=work_units, coherent_order=coherent_order, refill_min=refill_min,
              accuracy=_accuracy(geom, precision, accuracy))
    _check(lib.robast_trace_sources(geom.handle, src.handle, ctypes.c_uint64(seed & (2**64 - 1)),
                                    ctypes.c_void_p(group_counts.data_ptr()),
                                    ctypes.byref(tout) if tout is not None else None, ctypes.byref(o)))
    return group_counts


N_PARAM = 16
OBJECTIVES = {"msr": 0, "soft_ce": 1, "centroid_x": 2, "centroid_y": 3}


class ParamInfo(ctypes.Structure):
    _fields_ = [("surface", ctypes.c_int32), ("variant", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("active", ctypes.c_int32)]


PARAM_SLOTS = ("tilt_x", "tilt_y", "A1", "A2", "A3", "A4", "A5", "A6", "A7", "A8",
               "P0r", "P0z", "P1r", "P1z", "P2r", "P2z")


def param_layout(geom: Geometry):
    """robast_param_layout: per gradient parameter (surface, variant, slot name, active)."""
    lib = load()
    lib.robast_param_count.argtypes = [ctypes.c_void_p]
    lib.robast_param_layout.argtypes = [ctypes.c_void_p, ctypes.POINTER(ParamInfo)]
    n = lib.robast_param_count(geom.handle)
    arr = (ParamInfo * max(n, 1))()
    _check(lib.robast_param_layout(geom.handle, arr))
    return [(p.surface, p.variant, PARAM_SLOTS[p.slot], bool(p.active)) for p in arr[:n]]


def trace_grad(geom: Geometry, origins, dirs, wavelengths, objective="msr", seed: int = 0, precision: int = 32,
               tau: float = 0.5e-3, d_obj: float = 1.0, grad=True, max_bounces: int = 100, stream=None,
               variant_of_photon=None, first_photon_id: int = 0, eps: Optional[float] = None, out=None,
               work_units=None, coherent_order: int = 0):
    """robast_trace_grad: frozen-path objective value and d_obj * gradient.

    Returns (value, grad [n_surfaces, 16] float64 CUDA tensor or None, info dict).
    `out`, if given, is a float64 CUDA tensor [n_surfaces, 16] the gradient is added to.
    work_units: optional CUDA int64 tensor [>= 3], added to: FP64 interactions of the
    forward passes, interactions replayed by the reverse sweeps, dual-number interactions
    (the last two in the derivative precision: the trace's, or FP64 for geometries with cones).
    coherent_order: as for trace() (launch shape only; the sums are the same bits).
    """
    import torch
    lib = load()
    lib.robast_param_count.argtypes = [ctypes.c_void_p]
    lib.robast_trace_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                      ctypes.POINTER(TraceOpts), ctypes.POINTER(ctypes.c_double)]
    dt = torch.float32 if precision == 32 else torch.float64
    n = int(wavelengths.shape[0])
    for name, t, shape in (("origins", origins, (3, n)), ("dirs", dirs, (3, n)), ("wavelengths", wavelengths, (n,))):
        if t.dtype != dt or tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous():
            raise RobastError(f"{name}: need a contiguous CUDA {dt} tensor of shape {shape}")
    g = out
    if grad and g is None:
        g = torch.zeros((geom.n_surfaces, N_PARAM), dtype=torch.float64, device=origins.device)
    if stream is None:
        stream = torch.cuda.current_stream(origins.device)
    vop = ctypes.c_void_p(variant_of_photon.data_ptr()) if variant_of_photon is not None else None
    o = _opts(precision, max_bounces, ctypes.c_void_p(stream.cuda_stream), vop, first_photon_id, eps, 0, 0,
              units=work_units, coherent_order=coherent_order)
    val = ctypes.c_double()
    info = (ctypes.c_double * 8)()
    _check(lib.robast_trace_grad(geom.handle, _ptr(origins), _ptr(dirs), _ptr(wavelengths), n,
                                 ctypes.c_uint64(seed & (2**64 - 1)), OBJECTIVES[objective], float(tau), float(d_obj),
                                 ctypes.byref(val), ctypes.c_void_p(g.data_ptr()) if g is not None else None,
                                 ctypes.byref(o), info))
    keys = ("W", "sum_wqx", "sum_wqy", "sum_wq2", "sum_soft", "n_detected", "n_untracked", "n")
    res = dict(zip(keys, list(info)))
    if res["n_untracked"] > 0:
        import warnings
        warnings.warn(f"trace_grad: {int(res['n_untracked'])} photons contribute no gradient (a path longer than "
                      f"the adjoint's 64-interaction record, or a recomputed interaction that no longer met "
                      f"its surface)", RuntimeWarning)
    return val.value, g, res


def apply_params(scene, params):
    """A copy of `scene` with the 16 parameters per surface set from `params`
    ([n_surfaces, 16]: tilt x, y; A1..A8; Bezier P0r, P0z, P1r, P1z, P2r, P2z)."""
    import copy
    import numpy as np_
    p = np_.asarray(params, dtype=np_.float64).reshape(len(scene.surfaces), N_PARAM)
    sc = copy.copy(scene)
    sc.surfaces = []
    for s, row in zip(scene.surfaces, p):
        t = copy.copy(s)
        t.tilt = (float(row[0]), float(row[1]))
        if s.shape == "sag":
            t.asph = tuple(float(x) for x in row[2:10])
        if s.shape == "hexcone":
            t.prm = tuple(float(x) for x in row[10:16]) + tuple(s.prm[6:8])
        sc.surfaces.append(t)
    return sc


def scene_params(scene):
    """The [n_surfaces, 16] parameter array of a scene (see apply_params)."""
    import numpy as np_
    p = np_.zeros((len(scene.surfaces), N_PARAM))
    for i, s in enumerate(scene.surfaces):
        p[i, 0:2] = s.tilt
        p[i, 2:10] = list(s.asph) + [0.0] * (8 - len(s.asph))
        if s.shape == "hexcone":
            p[i, 10:16] = list(s.prm)[:6]
    return p


def objective_function():
    """torch.autograd.Function computing a frozen-path objective of a scene's
    parameters on the GPU; backward returns the gradient the same launch
    produced (scaled by the incoming gradient).

    Usage: FrozenPathObjective.apply(params, scene, origins, dirs, wavelengths, options_dict)
    with params a float64 tensor [n_surfaces, 16] (requires_grad).
    """
    import torch

    class FrozenPathObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, scene, origins, dirs, wavelengths, options):
            geom = build_geometry(apply_params(scene, params.detach().cpu().numpy()))
            value, grad, _ = trace_grad(geom, origins, dirs, wavelengths, **options)
            geom.close()
            ctx.save_for_backward(grad.to(params.device))
            return torch.tensor(value, dtype=torch.float64, device=params.device)

        @staticmethod
        def backward(ctx, grad_output):
            (grad,) = ctx.saved_tensors
            return grad_output * grad, None, None, None, None, None

    return FrozenPathObjective


def alloc_track(first: int, count: int, cap: int, precision: int = 32, device="cuda"):
    """Device buffers for photon-track recording (pass as trace(..., track=...))."""
    import torch
    dt = torch.float32 if precision == 32 else torch.float64
    return {"first": first, "count": count, "cap": cap,
            "points": torch.zeros((cap, 4), dtype=dt, device=device),
            "info": torch.zeros((cap, 4), dtype=torch.int32, device=device),
            "n_records": torch.zeros(1, dtype=torch.int64, device=device)}


def tracks_sorted(track):
    """Recorded tracks as numpy arrays sorted by (photon, bounce): points [k, 3], info [k, 4]."""
    import numpy as np_
    k = min(int(track["n_records"].item()), int(track["cap"]))
    pts = track["points"][:k, :3].cpu().numpy().astype(np_.float64)
    info = track["info"][:k].cpu().numpy()
    order = np_.lexsort((info[:, 1], info[:, 0]))
    return pts[order], info[order]
