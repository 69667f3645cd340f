"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
include/pxst.h declares; the binding covers them all. No compute calls here."""
import ctypes
import os
import re

import paper_2003_12726_gb300 as px

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "pxst.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pxst_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("pxst_make_object_map", "pxst_update_pixel_map", "pxst_iterate",
              "pxst_workspace_size", "pxst_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(px.library_path() if os.path.exists(px.library_path()) else px.lib()._name)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(px.EXPORTED) == sorted(n for n in declared() if n in px.EXPORTED)
    assert set(declared()) <= set(px.EXPORTED)


def test_host_only_calls():
    L = px.lib()
    assert L.pxst_status_string(0) == b"ok"
    assert b"sm_103a" in L.pxst_version()
    d = px.Dims(121, 512, 1536, 520, 1909)
    n = px.workspace_size(d, px.Options(1, 24))
    assert n > 16 * 520 * 1909
    assert px.workspace_size(px.Dims(0, 1, 1, 1, 1)) == 0
