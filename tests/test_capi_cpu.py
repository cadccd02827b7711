"""The C-ABI library without a GPU: it loads, it exports every entry point
declared in include/robast.h, and argument validation reports errors through
return codes and robast_last_error without aborting."""
import ctypes
import os
import re

import pytest

import paper_1508_07803_gb300 as robast
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "robast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(robast_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = robast.load()
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in robast.h but not exported"


def test_version_string():
    assert "sm_103a" in robast.version()


def _bad(scene_mut):
    scene = W.sphere_scene()
    scene_mut(scene)
    with pytest.raises(robast.RobastError) as ei:
        robast.build_geometry(scene)
    return str(ei.value)


def test_invalid_descriptors_are_rejected_with_messages():
    def bad_material(s):
        s.surfaces[0].material = 5
    assert "material" in _bad(bad_material)

    def bad_rot(s):
        s.surfaces[0].rot = (2, 0, 0, 0, 1, 0, 0, 0, 1)
    assert "orthonormal" in _bad(bad_rot)

    def bad_sector(s):
        s.surfaces[0].aperture = "sector"
        s.surfaces[0].ap = (0.1, 0.5, 0.0, 4.0)
    assert "sector" in _bad(bad_sector)

    def bad_scale(s):
        s.length_scale = 0.0
    assert "length_scale" in _bad(bad_scale)

    def bad_variants(s):
        s.variant_offsets = [0, 1]
    assert "variant_offsets" in _bad(bad_variants)

    def bad_asph(s):
        s.surfaces[0].aperture = "none"
        s.surfaces[0].asph = (1e-3,) + (0.0,) * 7
    assert "aspheric" in _bad(bad_asph)


def test_null_arguments_return_codes():
    lib = robast.load()
    assert lib.robast_build_geometry(None, None) == -2
    assert b"NULL" in lib.robast_last_error()
    assert lib.robast_trace(None, None, None, None, 0, 0, None) == -2
    lib.robast_free_geometry(None)  # ignored


def test_valid_descriptor_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(robast.RobastError) as ei:
        robast.build_geometry(W.lst_scene())
    assert "robast error -3" in str(ei.value) or "robast error -4" in str(ei.value)


_STRUCTS = {
    "robast_surface_desc": "SurfaceDesc", "robast_material_desc": "MaterialDesc", "robast_medium_desc": "MediumDesc",
    "robast_geom_desc": "GeomDesc", "robast_trace_out": "TraceOut", "robast_track_opts": "TrackOpts",
    "robast_trace_opts": "TraceOpts", "robast_source_group": "SourceGroupDesc", "robast_param_info": "ParamInfo",
}


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "robast.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        cls = getattr(robast, pyname)
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("    return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, pyname in _STRUCTS.items():
        cls = getattr(robast, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
