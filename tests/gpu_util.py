"""Helpers for the GPU tests: move a scan to the device and call the library through
its C ABI (via the Python binding)."""
from __future__ import annotations

import numpy as np

import paper_2003_12726_gb300 as px


def torch():
    import torch as t
    return t


def dev(a, dtype):
    t = torch()
    return t.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype).contiguous()


def dims_of(frames, ref_shape):
    n, ny, nx = frames.shape
    return px.Dims(int(n), int(ny), int(nx), int(ref_shape[0]), int(ref_shape[1]))


def gpu_make_object_map(frames, W, M, u, delta, ref_shape):
    t = torch()
    d = dims_of(frames, ref_shape)
    Iref = t.empty(ref_shape, dtype=t.float32, device="cuda")
    w = t.empty(ref_shape, dtype=t.float32, device="cuda")
    ws = px.workspace(d)
    px.make_object_map(d, dev(frames, t.float32), dev(W, t.float32), dev(M, t.uint8),
                       dev(u, t.float64), dev(delta, t.float64), Iref, w, ws)
    code, bits = px.get_status(ws)
    assert code == 0, (code, bits)
    return Iref.cpu().numpy(), w.cpu().numpy()


def gpu_update(frames, W, M, Iref32, w32, delta, u, window, quadratic=True, return_exact=False, form=0, tile=0):
    t = torch()
    d = dims_of(frames, Iref32.shape)
    o = px.Options(int(window[0]), int(window[1]), quadratic, form, tile=tile)
    ud = dev(u, t.float64)
    err = t.full(M.shape, -7.0, dtype=t.float32, device="cuda")
    ws = px.workspace(d, o)
    px.update_pixel_map(d, o, dev(frames, t.float32), dev(W, t.float32), dev(M, t.uint8),
                        dev(Iref32, t.float32), dev(w32, t.float32), dev(delta, t.float64), ud, err, ws)
    code, bits = px.get_status(ws)
    assert code == 0, (code, bits)
    n_exact = px.last_exact_count(ws)
    out = (ud.cpu().numpy(), err.cpu().numpy().astype(np.float64))
    return out + (n_exact,) if return_exact else out


def gpu_iterate(frames, W, M, delta, u, ref_shape, window, n_iter, quadratic=True, form=0):
    t = torch()
    d = dims_of(frames, ref_shape)
    o = px.Options(int(window[0]), int(window[1]), quadratic, form)
    ud = dev(u, t.float64)
    Iref = t.empty(ref_shape, dtype=t.float32, device="cuda")
    w = t.empty(ref_shape, dtype=t.float32, device="cuda")
    err = t.empty(M.shape, dtype=t.float32, device="cuda")
    ws = px.workspace(d, o)
    px.iterate(d, o, n_iter, dev(frames, t.float32), dev(W, t.float32), dev(M, t.uint8),
               dev(delta, t.float64), ud, Iref, w, err, ws)
    code, bits = px.get_status(ws)
    assert code == 0, (code, bits)
    return ud.cpu().numpy(), Iref.cpu().numpy(), w.cpu().numpy(), err.cpu().numpy().astype(np.float64)


def gpu_iteration_pair(s, u_start, form=0, tile=0):
    """One main-loop iteration (pxst_iterate, n_iter = 1) from u_start without and with the
    3x3 fit: two tuples (u, err, I_ref, w) for parity.check_iteration."""
    out = []
    for q in (False, True):
        t = torch()
        d = dims_of(s.frames, s.ref_shape)
        o = px.Options(int(s.window[0]), int(s.window[1]), q, form, tile=tile)
        ud = dev(u_start, t.float64)
        Iref = t.empty(s.ref_shape, dtype=t.float32, device="cuda")
        w = t.empty(s.ref_shape, dtype=t.float32, device="cuda")
        err = t.empty(s.M.shape, dtype=t.float32, device="cuda")
        ws = px.workspace(d, o)
        px.iterate(d, o, 1, dev(s.frames, t.float32), dev(s.W, t.float32), dev(s.M, t.uint8),
                   dev(s.delta, t.float64), ud, Iref, w, err, ws)
        code, bits = px.get_status(ws)
        assert code == 0, (code, bits)
        out.append((ud.cpu().numpy(), err.cpu().numpy().astype(np.float64), Iref.cpu().numpy(), w.cpu().numpy()))
    return out[0], out[1]
