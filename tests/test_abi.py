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


def _update_status(opts, dims=(16, 64, 64, 160, 160), frames=0x1000):
    """pxst_update_pixel_map with placeholder pointers and a zero-byte workspace: every call
    here is refused by the argument checks or, when the options pass, by the workspace size
    (PXST_ERR_NOMEM), before anything reaches the GPU."""
    L = px.lib()
    d = px._Dims(*dims)
    o = px._Opts(*opts)
    p = 0x100000
    return L.pxst_update_pixel_map(ctypes.byref(d), ctypes.byref(o), frames, p, p, p, p, p, p, None, 0x100000, 0,
                                   None)


def test_option_checks_fp32_tile_and_strip():
    ERR_ARG, ERR_SHAPE, ERR_NOMEM = -1, -2, -5
    # tile height (bits 0-3) and strip length (bits 4-5) of the FP32 form
    for tile in (0, 1, 2, 4, 8, 0x10, 0x11, 0x22, 0x34, 0x38):
        assert _update_status((4, 4, 1, 0, 0, tile, 0)) == ERR_NOMEM, hex(tile)
    for tile in (3, 5, 16 * 4, -1, 0x43, 0x17):
        assert _update_status((4, 4, 1, 0, 0, tile, 0)) == ERR_ARG, hex(tile)


def test_option_checks_tensor_forms_and_the_rest():
    ERR_ARG, ERR_SHAPE, ERR_NOMEM = -1, -2, -5
    for form in (1, 2):
        for tile in (0, 1, 2):
            assert _update_status((4, 4, 1, form, 0, tile, 0)) == ERR_NOMEM
        for tile in (3, 0x11):
            assert _update_status((4, 4, 1, form, 0, tile, 0)) == ERR_ARG
        for k in (4, 8):
            assert _update_status((4, 4, 1, form, k, 0, 0)) == ERR_NOMEM
        assert _update_status((4, 4, 1, form, 5, 0, 0)) == ERR_ARG
    assert _update_status((4, 4, 1, 3, 0, 0, 0)) == ERR_ARG              # unknown form
    assert _update_status((-1, 4, 1, 0, 0, 0, 0)) == ERR_ARG             # negative window
    assert _update_status((4, 4, 2, 0, 0, 0, 0)) == ERR_ARG              # quadratic not 0/1
    assert _update_status((4, 4, 1, 0, 0, 0, 0), dims=(0, 64, 64, 160, 160)) == ERR_SHAPE
    assert _update_status((4, 4, 1, 0, 0, 0, 0), frames=None) == ERR_ARG
