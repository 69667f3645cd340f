"""FP64 CPU oracle for the PXST hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (the CUDA library and its Python binding) never
imports it, and the two share no code.

The arithmetic lives in ``pxst_oracle.c`` (plain C, FP64, no fused multiply-add);
this module compiles it with gcc on first use and wraps it with numpy-friendly calls.
The paper sections each function follows are cited in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pxst_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpxst_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (seconds). Returns the shared-library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def default_threads():
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def _bind(L):
    i32, i64, dbl = C.c_int, C.c_int64, C.c_double
    P = C.c_void_p
    L.pxst_oracle_bilinear.argtypes = [dbl, dbl, C.POINTER(i64), C.POINTER(i64), P]
    L.pxst_oracle_gather.argtypes = [P, P, i64, i64, dbl, dbl, C.POINTER(dbl)]
    L.pxst_oracle_gather.restype = i32
    L.pxst_oracle_make_object_map.argtypes = [i32] * 5 + [P] * 7
    L.pxst_oracle_quadratic_fit.argtypes = [P, C.POINTER(dbl), C.POINTER(dbl)]
    L.pxst_oracle_pixel_window.argtypes = [i32] * 7 + [P] * 7 + [i64, P, P]
    L.pxst_oracle_update_pixel_map.argtypes = [i32] * 8 + [P] * 9 + [i32, i32, i32]
    L.pxst_oracle_update_pixels.argtypes = [i32] * 8 + [P] * 7 + [P, i64, P, P, i32]
    L.pxst_oracle_iterate.argtypes = [i32] * 9 + [P] * 7 + [P, i32]
    L.pxst_oracle_reference_terms.argtypes = [i32] * 3 + [P] * 5 + [i32]
    L.pxst_oracle_calc_error.argtypes = [i32] * 5 + [P] * 11
    L.pxst_oracle_frame_window.argtypes = [i32] * 7 + [P] * 7 + [i32, P]
    L.pxst_oracle_update_translations.argtypes = [i32] * 8 + [P] * 9
    L.pxst_oracle_filter_map.argtypes = [i32, i32, dbl, P, P, P]
    L.pxst_oracle_update_pixel_map_frac.argtypes = [i32] * 8 + [P] * 9 + [i32]
    L.pxst_oracle_contrast.argtypes = [i64, P, P]
    L.pxst_oracle_contrast.restype = dbl
    L.pxst_oracle_defocus_sweep.argtypes = [i32] * 5 + [P] * 5 + [i32, P, i32, P, P]
    L.pxst_oracle_integrate_map.argtypes = [i32, i32, P, P, i32, dbl, P, P]
    L.pxst_oracle_integrate_map.restype = i32
    return L


def lib():
    """The oracle library built from pxst_oracle.c."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def load_variant(so_path):
    """Wrap another build of the oracle source (the mutation tests plant a mistake in a
    copy of pxst_oracle.c and check that a pin catches it)."""
    return _bind(C.CDLL(so_path))


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


# ------------------------------------------------------------------------------------
def bilinear(a, b, L=None):
    """(i0, j0, weights[4]) of the point (a, b); weight order 00, 01, 10, 11."""
    i0, j0 = C.c_int64(), C.c_int64()
    w = np.zeros(4)
    (L or lib()).pxst_oracle_bilinear(float(a), float(b), C.byref(i0), C.byref(j0), _p(w))
    return i0.value, j0.value, w


def gather(Iref, w, q0, q1, L=None):
    """Masked renormalised bilinear read of I_ref at (q0, q1); None if invalid."""
    Iref, w = _f64(Iref), _f64(w)
    out = C.c_double()
    ok = (L or lib()).pxst_oracle_gather(_p(Iref), _p(w), Iref.shape[0], Iref.shape[1],
                                  float(q0), float(q1), C.byref(out))
    return out.value if ok else None


def make_object_map(frames, W, M, u, delta, ref_shape, L=None):
    """(I_ref, w), both float64 [Ry][Rx]."""
    frames, W, M, u, delta = _f32(frames), _f32(W), _u8(M), _f64(u), _f64(delta)
    N, ny, nx = frames.shape
    Ry, Rx = ref_shape
    Iref = np.empty((Ry, Rx))
    w = np.empty((Ry, Rx))
    (L or lib()).pxst_oracle_make_object_map(N, ny, nx, Ry, Rx, _p(frames), _p(W), _p(M), _p(u),
                                      _p(delta), _p(Iref), _p(w))
    return Iref, w


def quadratic_fit(f, L=None):
    """Sub-pixel shift (da, db) from the 3x3 errors f (da outer); inf = missing."""
    f = _f64(np.asarray(f).reshape(9))
    da, db = C.c_double(), C.c_double()
    (L or lib()).pxst_oracle_quadratic_fit(_p(f), C.byref(da), C.byref(db))
    return da.value, db.value


def pixel_window(frames, W, M, Iref, w, delta, u, window, p, L=None):
    """Normalised error over the whole window of flat pixel index p, and its centre."""
    frames, W, M, Iref, w, delta, u = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w),
                                       _f64(delta), _f64(u))
    N, ny, nx = frames.shape
    Sy, Sx = window
    e = np.empty((2 * Sy + 1, 2 * Sx + 1))
    centre = np.zeros(2, dtype=np.int64)
    (L or lib()).pxst_oracle_pixel_window(N, ny, nx, Iref.shape[0], Iref.shape[1], Sy, Sx, _p(frames),
                                   _p(W), _p(M), _p(Iref), _p(w), _p(delta), _p(u), int(p),
                                   _p(e), _p(centre))
    return e, (int(centre[0]), int(centre[1]))


def update_pixel_map(frames, W, M, Iref, w, delta, u, window, quadratic=True, rows=None,
                     threads=None, L=None):
    """(u_new [2][ny][nx], err [ny][nx]); only rows [r0, r1) are updated if given."""
    frames, W, M, Iref, w, delta = _f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w), _f64(delta)
    u_in = _f64(u)
    N, ny, nx = frames.shape
    Sy, Sx = window
    r0, r1 = rows if rows is not None else (0, ny)
    u_out = u_in.copy()
    err = np.full((ny, nx), np.nan)
    (L or lib()).pxst_oracle_update_pixel_map(N, ny, nx, Iref.shape[0], Iref.shape[1], Sy, Sx,
                                       int(bool(quadratic)), _p(frames), _p(W), _p(M), _p(Iref),
                                       _p(w), _p(delta), _p(u_in), _p(u_out), _p(err), int(r0),
                                       int(r1), int(threads or default_threads()))
    return u_out, err


def update_pixels(frames, W, M, Iref, w, delta, u, window, pix, quadratic=True, threads=None, L=None):
    """The update for a list of flat pixel indices: (u_new [K][2], err [K])."""
    frames, W, M, Iref, w, delta, u = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w),
                                       _f64(delta), _f64(u))
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    N, ny, nx = frames.shape
    Sy, Sx = window
    u_out = np.empty((pix.size, 2))
    err = np.empty(pix.size)
    (L or lib()).pxst_oracle_update_pixels(N, ny, nx, Iref.shape[0], Iref.shape[1], Sy, Sx,
                                    int(bool(quadratic)), _p(frames), _p(W), _p(M), _p(Iref),
                                    _p(w), _p(delta), _p(u), _p(pix), pix.size, _p(u_out),
                                    _p(err), int(threads or default_threads()))
    return u_out, err


def iterate(frames, W, M, delta, u, ref_shape, window, n_iter, quadratic=True, threads=None, L=None):
    """n_iter x (make_object_map, update_pixel_map): (u, I_ref, w, err)."""
    frames, W, M, delta = _f32(frames), _f32(W), _u8(M), _f64(delta)
    u = _f64(u).copy()
    N, ny, nx = frames.shape
    Ry, Rx = ref_shape
    Sy, Sx = window
    Iref = np.zeros((Ry, Rx))
    w = np.zeros((Ry, Rx))
    err = np.full((ny, nx), np.nan)
    (L or lib()).pxst_oracle_iterate(N, ny, nx, Ry, Rx, Sy, Sx, int(bool(quadratic)), int(n_iter),
                              _p(frames), _p(W), _p(M), _p(delta), _p(u), _p(Iref), _p(w),
                              _p(err), int(threads or default_threads()))
    return u, Iref, w, err


def reference_terms(Iref, w, delta, threads=None, L=None):
    """(T float64 [Ry][Rx], nvalid int32 [Ry][Rx]): sum_n V R^2 and sum_n V."""
    Iref, w, delta = _f64(Iref), _f64(w), _f64(delta)
    Ry, Rx = Iref.shape
    T = np.empty((Ry, Rx))
    nv = np.empty((Ry, Rx), dtype=np.int32)
    (L or lib()).pxst_oracle_reference_terms(delta.shape[0], Ry, Rx, _p(Iref), _p(w), _p(delta),
                                             _p(T), _p(nv), int(threads or default_threads()))
    return T, nv


def calc_error(frames, W, M, Iref, w, u, delta, L=None):
    """Figures of merit (section "Calculate figures of merit"): (pixel error [ny][nx] (NaN
    where M = 0), frame error [N], total error, reference-plane error [Ry][Rx])."""
    frames, W, M, Iref, w, u, delta = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w), _f64(u),
                                       _f64(delta))
    N, ny, nx = frames.shape
    Ry, Rx = Iref.shape
    pe = np.empty((ny, nx))
    fe = np.empty(N)
    tot = np.zeros(1)
    re = np.empty((Ry, Rx))
    (L or lib()).pxst_oracle_calc_error(N, ny, nx, Ry, Rx, _p(frames), _p(W), _p(M), _p(Iref), _p(w), _p(u),
                                        _p(delta), _p(pe), _p(fe), _p(tot), _p(re))
    return pe, fe, float(tot[0]), re


def frame_window(frames, W, M, Iref, w, u, delta, twindow, n, L=None):
    """Error of frame n over the window of integer shifts of its translation."""
    frames, W, M, Iref, w, u, delta = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w), _f64(u),
                                       _f64(delta))
    N, ny, nx = frames.shape
    Ty, Tx = twindow
    e = np.empty((2 * Ty + 1, 2 * Tx + 1))
    (L or lib()).pxst_oracle_frame_window(N, ny, nx, Iref.shape[0], Iref.shape[1], Ty, Tx, _p(frames), _p(W),
                                          _p(M), _p(Iref), _p(w), _p(u), _p(delta), int(n), _p(e))
    return e


def update_translations(frames, W, M, Iref, w, u, delta, twindow, quadratic=True, L=None):
    """Section "Update translations": (new translations [N][2], each frame's error at its
    argmin [N])."""
    frames, W, M, Iref, w, u, delta = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w), _f64(u),
                                       _f64(delta))
    N, ny, nx = frames.shape
    Ty, Tx = twindow
    d_out = np.empty((N, 2))
    err = np.empty(N)
    (L or lib()).pxst_oracle_update_translations(N, ny, nx, Iref.shape[0], Iref.shape[1], Ty, Tx,
                                                 int(bool(quadratic)), _p(frames), _p(W), _p(M), _p(Iref),
                                                 _p(w), _p(u), _p(delta), _p(d_out), _p(err))
    return d_out, err


def filter_map(M, u, sigma, L=None):
    """The "sigma" regularisation of the pixel map: Gaussian filter normalised over the good
    pixels (M = 0 pixels keep u)."""
    M, u = _u8(M), _f64(u)
    ny, nx = M.shape
    out = np.empty_like(u)
    (L or lib()).pxst_oracle_filter_map(ny, nx, float(sigma), _p(M), _p(u), _p(out))
    return out


def update_pixel_map_frac(frames, W, M, Iref, w, delta, u, window, sub, threads=None, L=None):
    """The non-integer candidate option: the integer search, then the candidates on a 1/sub
    grid within one pixel of its minimum: (u_new [2][ny][nx], err [ny][nx])."""
    frames, W, M, Iref, w, delta, u = (_f32(frames), _f32(W), _u8(M), _f64(Iref), _f64(w), _f64(delta), _f64(u))
    N, ny, nx = frames.shape
    Sy, Sx = window
    u_out = u.copy()
    err = np.full((ny, nx), np.nan)
    (L or lib()).pxst_oracle_update_pixel_map_frac(N, ny, nx, Iref.shape[0], Iref.shape[1], Sy, Sx, int(sub),
                                                   _p(frames), _p(W), _p(M), _p(Iref), _p(w), _p(delta), _p(u),
                                                   _p(u_out), _p(err), int(threads or default_threads()))
    return u_out, err


def contrast(Iref, w, L=None):
    """Standard deviation over mean of I_ref over the pixels with w > 0."""
    Iref, w = _f64(Iref), _f64(w)
    return float((L or lib()).pxst_oracle_contrast(Iref.size, _p(Iref), _p(w)))


def defocus_sweep(frames, W, M, u, delta, ref_shape, sy, sx, L=None):
    """fit_defocus_registration: the contrast of the reference image for each pair of map
    scales (sy[ky], sx[kx]) about the detector's central pixel: [len(sy)][len(sx)]."""
    frames, W, M, u, delta = _f32(frames), _f32(W), _u8(M), _f64(u), _f64(delta)
    sy, sx = _f64(sy), _f64(sx)
    N, ny, nx = frames.shape
    out = np.empty((sy.size, sx.size))
    (L or lib()).pxst_oracle_defocus_sweep(N, ny, nx, ref_shape[0], ref_shape[1], _p(frames), _p(W), _p(M), _p(u),
                                           _p(delta), sy.size, _p(sy), sx.size, _p(sx), _p(out))
    return out


def integrate_map(M, u, max_iter=100000, tol=1e-12, L=None):
    """The "integrate" option (R17): least-squares integration of the map u [2][ny][nx] over
    the good pixels by conjugate gradients and re-differentiation. Returns (u_out, steps,
    relative residual)."""
    L = L or lib()
    ny, nx = M.shape
    Mu = _u8(M)
    uin = _f64(u)
    out = np.empty_like(uin)
    res = C.c_double(0.0)
    it = L.pxst_oracle_integrate_map(ny, nx, _p(Mu), _p(uin), int(max_iter), float(tol), _p(out), C.byref(res))
    return out, int(it), float(res.value)
