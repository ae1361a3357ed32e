"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gbfwi.h declares; host-only calls behave without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2009_12663_gb300 as gb
from paper_2009_12663_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gbfwi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbfwi_[a-z0-9_]+)\s*\(", txt)))


def test_header_lists_match_binding():
    assert sorted(_lib.ABI_SYMBOLS) == _declared()


def test_library_exports_every_declared_symbol():
    L = gb.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_library_is_sm103a_and_in_tree():
    from paper_2009_12663_gb300 import build
    path = build.build()
    assert os.path.commonpath([path, ROOT]) == ROOT
    assert "compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror_and_tiles_host_only():
    L = gb.lib()
    assert L.gbfwi_strerror(0) == b"ok"
    assert b"curvature" in L.gbfwi_strerror(-5)
    assert L.gbfwi_strerror(12345) == b"unknown error"
    assert gb.num_tiles() >= 1
    for t in range(gb.num_tiles()):
        tx, tz = gb.tile_shape(t)
        assert tx >= 1 and tz >= 1 and ((tx + 1) * (tz + 1)) % 32 == 0
    with pytest.raises(gb.GbfwiError):
        gb.tile_shape(gb.num_tiles())


def test_mesh_create_rejects_bad_arguments_before_any_device_call():
    src = [dict(x=10.0, z=10.0, type=0, f0=10.0)]
    rec = np.array([[5.0, 0.0]])
    bad = [
        dict(nex=0, nez=4, h=10.0, dt=1e-3, nt=10),      # no elements
        dict(nex=4, nez=4, h=-1.0, dt=1e-3, nt=10),      # negative size
        dict(nex=4, nez=4, h=10.0, dt=0.0, nt=10),       # zero dt
        dict(nex=4, nez=4, h=10.0, dt=1e-3, nt=1),       # too few steps
    ]
    for kw in bad:
        with pytest.raises(gb.GbfwiError) as e:
            gb.Mesh(kw["nex"], kw["nez"], kw["h"], kw["dt"], kw["nt"], src, rec)
        assert e.value.name == "EINVAL"
    # source outside the mesh
    with pytest.raises(gb.GbfwiError) as e:
        gb.Mesh(4, 4, 10.0, 1e-3, 10, [dict(x=100.0, z=10.0, f0=10.0)], rec)
    assert e.value.name == "EINVAL"
    # bad source type
    with pytest.raises(gb.GbfwiError) as e:
        gb.Mesh(4, 4, 10.0, 1e-3, 10, [dict(x=10.0, z=10.0, type=7, f0=10.0)], rec)
    assert e.value.name == "EINVAL"


def test_null_handles_rejected():
    L = gb.lib()
    assert L.gbfwi_mesh_dims(None, None, None) == -1
    assert L.gbfwi_bfgs_count(None) == -1
    assert L.gbfwi_forward(None, None, 0, None, None) == -1
    assert L.gbfwi_bfgs_apply(None, None, 1, None, ctypes.c_double(1.0), 0, None) == -1
    assert L.gbfwi_mesh_destroy(None) == 0
    assert L.gbfwi_bfgs_destroy(None) == 0


def test_foreign_device_pointer_is_rejected_by_the_pointer_rule(tmp_path):
    """The rule every entry point applies to its array arguments
    (csrc/ptrclass.h), compiled with the host C compiler and fed the pointer
    attributes a GPU would report: device memory of another device than the
    current one is rejected, memory of the current device is used in place,
    managed memory is reachable from any device, host memory is staged."""
    src = tmp_path / "ptr.c"
    src.write_text(
        '#include <stdio.h>\n#include "ptrclass.h"\n'
        "int main(void) {\n"
        "  int cases[][4] = {\n"
        "    {GB_MEMTYPE_DEVICE, 1, 0, GB_PTR_FOREIGN}, {GB_MEMTYPE_DEVICE, 0, 1, GB_PTR_FOREIGN},\n"
        "    {GB_MEMTYPE_DEVICE, 3, 3, GB_PTR_LOCAL}, {GB_MEMTYPE_MANAGED, 2, 0, GB_PTR_LOCAL},\n"
        "    {GB_MEMTYPE_HOST, 1, 0, GB_PTR_HOST}, {GB_MEMTYPE_UNREGISTERED, -2, 0, GB_PTR_HOST},\n"
        "    {GB_MEMTYPE_DEVICE, 0, -1, GB_PTR_FOREIGN}};\n"
        "  int bad = 0;\n"
        "  for (unsigned i = 0; i < sizeof cases / sizeof cases[0]; ++i)\n"
        "    if (gb_classify_pointer(cases[i][0], cases[i][1], cases[i][2]) != cases[i][3]) { printf(\"%u\\n\", i); bad = 1; }\n"
        "  return bad;\n}\n")
    exe = tmp_path / "ptr"
    import subprocess
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I",
                           os.path.join(ROOT, "paper_2009_12663_gb300", "csrc"), str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
