"""Python binding of libpxst.so, the GB300 PXST hot-path library (see include/pxst.h).

Argument marshalling only: every step of make_object_map / update_pixel_map / iterate
runs in the library's CUDA kernels. PyTorch supplies device memory and the stream.
There is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

Tensor conventions (all CUDA, C-contiguous):
    frames float32 [N][ny][nx], W float32 [ny][nx], M uint8 [ny][nx],
    u float64 [2][ny][nx], delta float64 [N][2], I_ref / w float32 [Ry][Rx].
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

STATUS = {0: "ok", -1: "invalid argument", -2: "invalid shape", -3: "range", -4: "cuda error",
          -5: "workspace too small", -6: "timeout", -7: "bad input"}
FORM_FP32 = 0
FORM_BF16 = 1
FORM_TF32 = 2
KERNELS = ["prepare", "omap_scatter", "omap_normalise", "upm_search", "upm_exact", "reference_terms",
           "tensor_prep", "tensor_gtable", "tensor_search", "upm_rescore", "calc_error",
           "update_translations", "filter_map", "upm_fractional", "defocus_sweep", "integrate"]


class PxstError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"pxst: {what} failed with status {code} ({STATUS.get(code, '?')})")


class _Dims(C.Structure):
    _fields_ = [("n_frames", C.c_int32), ("ny", C.c_int32), ("nx", C.c_int32),
                ("ref_ny", C.c_int32), ("ref_nx", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("win_y", C.c_int32), ("win_x", C.c_int32), ("quadratic", C.c_int32),
                ("form", C.c_int32), ("rescore_k", C.c_int32), ("tile", C.c_int32),
                ("timeout_ns", C.c_int64)]


class _Scan(C.Structure):
    _fields_ = [("dims", _Dims), ("opts", _Opts), ("frames", C.c_void_p), ("W", C.c_void_p),
                ("mask", C.c_void_p), ("delta", C.c_void_p), ("u", C.c_void_p), ("I_ref", C.c_void_p),
                ("w", C.c_void_p), ("err_out", C.c_void_p), ("workspace", C.c_void_p),
                ("ws_bytes", C.c_size_t)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libpxst.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpxst.so is missing: the CUDA extension was not built")
        L = C.CDLL(path)
        P, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        D, O = C.POINTER(_Dims), C.POINTER(_Opts)
        L.pxst_workspace_size.argtypes = [D, O]
        L.pxst_workspace_size.restype = sz
        L.pxst_make_object_map.argtypes = [D] + [P] * 8 + [sz, P]
        L.pxst_make_object_map.restype = i32
        L.pxst_make_object_map_noalloc.argtypes = [D] + [P] * 8
        L.pxst_make_object_map_noalloc.restype = i32
        L.pxst_update_pixel_map.argtypes = [D, O] + [P] * 9 + [sz, P]
        L.pxst_update_pixel_map.restype = i32
        L.pxst_iterate.argtypes = [D, O, i32] + [P] * 9 + [sz, P]
        L.pxst_iterate.restype = i32
        L.pxst_reference_terms.argtypes = [D] + [P] * 6 + [sz, P]
        L.pxst_reference_terms.restype = i32
        L.pxst_get_status.argtypes = [P, P, C.POINTER(i32)]
        L.pxst_get_status.restype = i32
        L.pxst_last_exact_count.argtypes = [P, P, C.POINTER(i64)]
        L.pxst_last_exact_count.restype = i32
        L.pxst_timing_enable.argtypes = [i32]
        L.pxst_timing_enable.restype = i32
        L.pxst_timing_read.argtypes = [C.POINTER(i64), C.POINTER(C.c_double), i32]
        L.pxst_timing_read.restype = i32
        L.pxst_kernel_name.argtypes = [i32]
        L.pxst_kernel_name.restype = C.c_char_p
        L.pxst_status_string.argtypes = [i32]
        L.pxst_status_string.restype = C.c_char_p
        L.pxst_version.restype = C.c_char_p
        L.pxst_launch_count.argtypes = [C.POINTER(i64)]
        L.pxst_launch_count.restype = i32
        L.pxst_wait_flag.argtypes = [P, i32, i64, P, sz, P]
        L.pxst_wait_flag.restype = i32
        L.pxst_integrate_map.argtypes = [D, P, P, i32, C.c_double, i64, P, P, sz, P]
        L.pxst_integrate_map.restype = i32
        L.pxst_tensor_check.argtypes = [i32, i32, P, P, P, P, P]
        L.pxst_tensor_check.restype = i32
        S = C.POINTER(_Scan)
        L.pxst_batch_plan.argtypes = [S, i32, i32, i32, i32, P, C.POINTER(P)]
        L.pxst_batch_plan.restype = i32
        L.pxst_batch_run.argtypes = [P, P]
        L.pxst_batch_run.restype = i32
        L.pxst_batch_branch.argtypes = [P, i32]
        L.pxst_batch_branch.restype = i32
        L.pxst_batch_destroy.argtypes = [P]
        L.pxst_batch_destroy.restype = None
        L.pxst_autotune.argtypes = [S, i32, P, C.POINTER(i32), C.POINTER(C.c_float)]
        L.pxst_autotune.restype = i32
        L.pxst_calc_error.argtypes = [D] + [P] * 12 + [sz, P]
        L.pxst_calc_error.restype = i32
        L.pxst_update_translations.argtypes = [D, i32, i32, i32] + [P] * 9 + [sz, P]
        L.pxst_update_translations.restype = i32
        L.pxst_filter_map.argtypes = [D, C.c_double, P, P, P, sz, P]
        L.pxst_filter_map.restype = i32
        L.pxst_update_pixel_map_fractional.argtypes = [D, O, i32] + [P] * 9 + [sz, P]
        L.pxst_update_pixel_map_fractional.restype = i32
        L.pxst_defocus_sweep.argtypes = [D] + [P] * 5 + [i32, P, i32, P] + [P] * 4 + [sz, P]
        L.pxst_defocus_sweep.restype = i32
        _lib = L
    return _lib


EXPORTED = ["pxst_workspace_size", "pxst_make_object_map", "pxst_make_object_map_noalloc",
            "pxst_update_pixel_map",
            "pxst_iterate", "pxst_reference_terms", "pxst_get_status", "pxst_last_exact_count",
            "pxst_timing_enable", "pxst_timing_read", "pxst_kernel_name", "pxst_status_string",
            "pxst_version", "pxst_tensor_check", "pxst_batch_plan", "pxst_batch_run", "pxst_batch_branch",
            "pxst_batch_destroy", "pxst_autotune", "pxst_calc_error", "pxst_update_translations",
            "pxst_filter_map", "pxst_update_pixel_map_fractional", "pxst_defocus_sweep", "pxst_launch_count",
            "pxst_wait_flag", "pxst_integrate_map"]


# ---------------------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _check(t, dtype, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _ptr_or_null(t, dtype, shape, name):
    return C.c_void_p(None) if t is None else _check(t, dtype, shape, name)


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class Dims:
    n_frames: int
    ny: int
    nx: int
    ref_ny: int
    ref_nx: int

    def c(self):
        return _Dims(self.n_frames, self.ny, self.nx, self.ref_ny, self.ref_nx)


@dataclass
class Options:
    win_y: int
    win_x: int
    quadratic: bool = True
    form: int = FORM_FP32
    rescore_k: int = 0      # tensor forms: 4 or 8 (0: 8 below 128 frames, else 4)
    tile: int = 0           # tile shape (0: automatic); see pxst_options.tile
    timeout_ns: int = 0     # limit of the device-side waits (0: 1 s)

    def c(self):
        return _Opts(self.win_y, self.win_x, 1 if self.quadratic else 0, self.form, self.rescore_k, self.tile,
                     self.timeout_ns)


def workspace_size(dims: Dims, opts: Options | None = None):
    o = opts.c() if opts is not None else None
    return int(lib().pxst_workspace_size(C.byref(dims.c()), C.byref(o) if o is not None else None))


def workspace(dims: Dims, opts: Options | None = None, device=None):
    """A caller-owned workspace tensor (uint8, 256-byte aligned by the torch allocator)."""
    torch = _torch()
    n = workspace_size(dims, opts)
    if n == 0:
        raise PxstError(-2, "workspace_size")
    ws = torch.zeros(n, dtype=torch.uint8, device=device or "cuda")
    assert ws.data_ptr() % 256 == 0
    return ws


def _raise(code, what):
    if code != 0:
        raise PxstError(code, what)


def make_object_map(dims: Dims, frames, W, M, u, delta, I_ref, w, ws, stream=None):
    """pxst_make_object_map: fills I_ref and w (float32 [Ry][Rx])."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    args = [_check(frames, torch.float32, (N, ny, nx), "frames"), _check(W, torch.float32, (ny, nx), "W"),
            _check(M, torch.uint8, (ny, nx), "M"), _check(u, torch.float64, (2, ny, nx), "u"),
            _check(delta, torch.float64, (N, 2), "delta"), _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
            _check(w, torch.float32, (Ry, Rx), "w")]
    _raise(lib().pxst_make_object_map(C.byref(dims.c()), *args, C.c_void_p(ws.data_ptr()), ws.numel(),
                                      _stream(stream)), "make_object_map")


def make_object_map_noalloc(dims: Dims, frames, W, M, u, delta, I_ref, w, stream=None):
    """pxst_make_object_map_noalloc: as make_object_map, for callers that cannot allocate
    device memory (its scratch is a fixed array inside the library; at most 8192 frames and
    1048576 reference pixels; calls that overlap on the GPU race)."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    args = [_check(frames, torch.float32, (N, ny, nx), "frames"), _check(W, torch.float32, (ny, nx), "W"),
            _check(M, torch.uint8, (ny, nx), "M"), _check(u, torch.float64, (2, ny, nx), "u"),
            _check(delta, torch.float64, (N, 2), "delta"), _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
            _check(w, torch.float32, (Ry, Rx), "w")]
    _raise(lib().pxst_make_object_map_noalloc(C.byref(dims.c()), *args, _stream(stream)),
           "make_object_map_noalloc")


def update_pixel_map(dims: Dims, opts: Options, frames, W, M, I_ref, w, delta, u, err=None, ws=None,
                     stream=None):
    """pxst_update_pixel_map: updates u (float64 [2][ny][nx]) in place; err optional."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    args = [_check(frames, torch.float32, (N, ny, nx), "frames"), _check(W, torch.float32, (ny, nx), "W"),
            _check(M, torch.uint8, (ny, nx), "M"), _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
            _check(w, torch.float32, (Ry, Rx), "w"), _check(delta, torch.float64, (N, 2), "delta"),
            _check(u, torch.float64, (2, ny, nx), "u"), _ptr_or_null(err, torch.float32, (ny, nx), "err")]
    _raise(lib().pxst_update_pixel_map(C.byref(dims.c()), C.byref(opts.c()), *args,
                                       C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "update_pixel_map")


def iterate(dims: Dims, opts: Options, n_iter, frames, W, M, delta, u, I_ref, w, err=None, ws=None,
            stream=None):
    """pxst_iterate: n_iter x (make_object_map, update_pixel_map), all on the device."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    args = [_check(frames, torch.float32, (N, ny, nx), "frames"), _check(W, torch.float32, (ny, nx), "W"),
            _check(M, torch.uint8, (ny, nx), "M"), _check(delta, torch.float64, (N, 2), "delta"),
            _check(u, torch.float64, (2, ny, nx), "u"), _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
            _check(w, torch.float32, (Ry, Rx), "w"), _ptr_or_null(err, torch.float32, (ny, nx), "err")]
    _raise(lib().pxst_iterate(C.byref(dims.c()), C.byref(opts.c()), int(n_iter), *args,
                              C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)), "iterate")


def reference_terms(dims: Dims, I_ref, w, delta, T, n_valid, ws, stream=None):
    """pxst_reference_terms: T = sum_n V R^2 (float32) and n_valid = sum_n V (int32)."""
    torch = _torch()
    N, Ry, Rx = dims.n_frames, dims.ref_ny, dims.ref_nx
    args = [_check(I_ref, torch.float32, (Ry, Rx), "I_ref"), _check(w, torch.float32, (Ry, Rx), "w"),
            _check(delta, torch.float64, (N, 2), "delta"), _check(T, torch.float32, (Ry, Rx), "T"),
            _check(n_valid, torch.int32, (Ry, Rx), "n_valid")]
    _raise(lib().pxst_reference_terms(C.byref(dims.c()), *args, C.c_void_p(ws.data_ptr()), ws.numel(),
                                      _stream(stream)), "reference_terms")


def get_status(ws, stream=None):
    """(status code, raw device bits); synchronises the stream and clears the bits."""
    bits = C.c_int32()
    code = lib().pxst_get_status(C.c_void_p(ws.data_ptr()), _stream(stream), C.byref(bits))
    return int(code), int(bits.value)


def last_exact_count(ws, stream=None):
    n = C.c_int64()
    _raise(lib().pxst_last_exact_count(C.c_void_p(ws.data_ptr()), _stream(stream), C.byref(n)),
           "last_exact_count")
    return int(n.value)


def timing_enable(on=True):
    _raise(lib().pxst_timing_enable(1 if on else 0), "timing_enable")


def timing_read():
    """{kernel name: (launches, total ms)} since timing_enable(True)."""
    k = len(KERNELS)
    n = (C.c_int64 * k)()
    t = (C.c_double * k)()
    _raise(lib().pxst_timing_read(n, t, k), "timing_read")
    return {KERNELS[i]: (int(n[i]), float(t[i])) for i in range(k)}


def version():
    return lib().pxst_version().decode()


def wait_flag(flag, target, timeout_ns, ws, stream=None):
    """pxst_wait_flag: the work queued on `stream` after this call runs once the int32 at
    `flag` (a CUDA tensor, or a pinned CPU tensor, which the GPU reads through unified
    addressing) is >= target; gives up after timeout_ns (the status then reports a timeout)."""
    torch = _torch()
    if not isinstance(flag, torch.Tensor) or flag.dtype != torch.int32 or flag.numel() < 1:
        raise TypeError("flag must be an int32 tensor")
    if not flag.is_cuda and not flag.is_pinned():
        raise ValueError("flag must be on a CUDA device or in pinned host memory")
    _raise(lib().pxst_wait_flag(C.c_void_p(flag.data_ptr()), int(target), int(timeout_ns), C.c_void_p(ws.data_ptr()),
                                ws.numel(), _stream(stream)), "wait_flag")


def launch_count():
    """Kernel launches this library has issued in the process so far (pxst_launch_count)."""
    n = C.c_int64()
    _raise(lib().pxst_launch_count(C.byref(n)), "launch_count")
    return int(n.value)


# ---------------------------------------------------------------------------------------
class Reconstruction:
    """Device-resident state of one scan (frames, whitefield, mask, translations, map,
    reference image and workspace), for callers that hold their data on the host.

    ``run(n_iter)`` executes the main loop on the GPU; ``run_host`` is the end-to-end
    form: it copies the inputs from pinned host memory, iterates and copies the map
    and the error back, all on one stream.
    """

    def __init__(self, frames, W, M, delta, u, ref_shape, window, quadratic=True, device="cuda", form=FORM_FP32):
        torch = _torch()
        self.dims = Dims(int(frames.shape[0]), int(frames.shape[1]), int(frames.shape[2]),
                         int(ref_shape[0]), int(ref_shape[1]))
        self.opts = Options(int(window[0]), int(window[1]), bool(quadratic), int(form))
        dev = torch.device(device)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt).contiguous()
        self.frames = t(frames, torch.float32)
        self.W = t(W, torch.float32)
        self.M = t(M, torch.uint8)
        self.delta = t(delta, torch.float64)
        self.u = t(u, torch.float64)
        Ry, Rx = ref_shape
        self.I_ref = torch.zeros((Ry, Rx), dtype=torch.float32, device=dev)
        self.w = torch.zeros((Ry, Rx), dtype=torch.float32, device=dev)
        self.err = torch.zeros((self.dims.ny, self.dims.nx), dtype=torch.float32, device=dev)
        self.ws = workspace(self.dims, self.opts, dev)
        self._pinned = None

    @classmethod
    def from_device(cls, frames, W, M, delta, u, ref_shape, window, quadratic=True, form=FORM_FP32, tile=0):
        """State around inputs already on the device (the tensors are used as they are; u is
        cloned, so the caller's initial map is kept)."""
        torch = _torch()
        self = cls.__new__(cls)
        n, ny, nx = (int(v) for v in frames.shape)
        self.dims = Dims(n, ny, nx, int(ref_shape[0]), int(ref_shape[1]))
        self.opts = Options(int(window[0]), int(window[1]), bool(quadratic), int(form), tile=int(tile))
        dev = frames.device
        _check(frames, torch.float32, (n, ny, nx), "frames")
        _check(W, torch.float32, (ny, nx), "W")
        _check(M, torch.uint8, (ny, nx), "M")
        _check(delta, torch.float64, (n, 2), "delta")
        _check(u, torch.float64, (2, ny, nx), "u")
        self.frames, self.W, self.M, self.delta, self.u = frames, W, M, delta, u.clone()
        self.I_ref = torch.zeros(tuple(int(v) for v in ref_shape), dtype=torch.float32, device=dev)
        self.w = torch.zeros_like(self.I_ref)
        self.err = torch.zeros((ny, nx), dtype=torch.float32, device=dev)
        self.ws = workspace(self.dims, self.opts, dev)
        self._pinned = None
        return self

    def device_bytes(self):
        """Bytes of device memory this scan holds (inputs, state and workspace)."""
        ts = (self.frames, self.W, self.M, self.delta, self.u, self.I_ref, self.w, self.err, self.ws)
        return sum(t.numel() * t.element_size() for t in ts)

    def run(self, n_iter, stream=None):
        iterate(self.dims, self.opts, n_iter, self.frames, self.W, self.M, self.delta, self.u,
                self.I_ref, self.w, self.err, self.ws, stream)

    def pin_host_buffers(self, frames, W, M, delta, u):
        """Pinned host copies of the per-step inputs and the outputs (for run_host)."""
        torch = _torch()
        pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dt).pin_memory()
        self._pinned = dict(frames=pin(frames, torch.float32), W=pin(W, torch.float32),
                            M=pin(M, torch.uint8), delta=pin(delta, torch.float64), u=pin(u, torch.float64),
                            u_out=torch.empty((2, self.dims.ny, self.dims.nx), dtype=torch.float64).pin_memory(),
                            err_out=torch.empty((self.dims.ny, self.dims.nx), dtype=torch.float32).pin_memory())
        return self._pinned

    def run_host(self, n_iter, stream=None):
        """Host -> device inputs, n_iter iterations, device -> host map and error.
        Returns (h2d bytes, d2h bytes); the host results are in the pinned buffers."""
        torch = _torch()
        h = self._pinned
        s = stream or torch.cuda.current_stream()
        with torch.cuda.stream(s):
            for k in ("frames", "W", "M", "delta", "u"):
                getattr(self, k).copy_(h[k], non_blocking=True)
            self.run(n_iter, s)
            h["u_out"].copy_(self.u, non_blocking=True)
            h["err_out"].copy_(self.err, non_blocking=True)
        h2d = sum(h[k].numel() * h[k].element_size() for k in ("frames", "W", "M", "delta", "u"))
        d2h = h["u_out"].numel() * 8 + h["err_out"].numel() * 4
        return h2d, d2h


class HostStream:
    """Many steps of one scan fed from pinned host memory, end to end: every step copies its
    inputs (frames, whitefield, mask, translations, initial map) host to device, iterates, and
    copies the map and the error back. Two device input buffers alternate, so that step k+1's
    host-to-device copy (on a copy stream) runs while step k computes (on the compute stream);
    the reference image, error and workspace of `rec` serve every step, in order."""

    def __init__(self, rec, pinned):
        torch = _torch()
        self.rec = rec
        self.h = pinned
        self.copy = torch.cuda.Stream()
        self.compute = torch.cuda.Stream()
        mk = lambda t: torch.empty_like(t)
        self.bufs = [dict(frames=rec.frames, W=rec.W, M=rec.M, delta=rec.delta, u=rec.u),
                     dict(frames=mk(rec.frames), W=mk(rec.W), M=mk(rec.M), delta=mk(rec.delta), u=mk(rec.u))]
        self.copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]
        for e in self.done:
            e.record(self.compute)
        self.k = 0
        self.h2d = sum(pinned[k].numel() * pinned[k].element_size() for k in ("frames", "W", "M", "delta", "u"))
        self.d2h = pinned["u_out"].numel() * 8 + pinned["err_out"].numel() * 4

    def run(self, steps, n_iter=1):
        """`steps` end-to-end steps; returns on the host at once (work is queued). Per step:
        (h2d bytes, d2h bytes) = (self.h2d, self.d2h)."""
        torch = _torch()
        r = self.rec
        for _ in range(steps):
            k = self.k                                            # steps alternate buffers across calls
            self.k += 1
            b = self.bufs[k & 1]
            self.copy.wait_event(self.done[k & 1])                # the buffer's previous step is done
            with torch.cuda.stream(self.copy):
                for key in ("frames", "W", "M", "delta", "u"):
                    b[key].copy_(self.h[key], non_blocking=True)
                self.copied[k & 1].record(self.copy)
            self.compute.wait_event(self.copied[k & 1])
            with torch.cuda.stream(self.compute):
                iterate(r.dims, r.opts, n_iter, b["frames"], b["W"], b["M"], b["delta"], b["u"], r.I_ref, r.w,
                        r.err, r.ws, self.compute)
                self.h["u_out"].copy_(b["u"], non_blocking=True)
                self.h["err_out"].copy_(r.err, non_blocking=True)
                self.done[k & 1].record(self.compute)
        return self.h2d, self.d2h

    def synchronize(self):
        self.compute.synchronize()
        self.copy.synchronize()


def tensor_check(form, A, B, stream=None):
    """pxst_tensor_check: D = A . B^T on the tensor cores (A [128][K], B [256][K], CUDA
    tensors of bfloat16 for FORM_BF16 or float32 for FORM_TF32). Returns (D, status bits)."""
    torch = _torch()
    K = int(A.shape[1])
    dt = torch.bfloat16 if form == FORM_BF16 else torch.float32
    a = _check(A, dt, (128, K), "A")
    b = _check(B, dt, (256, K), "B")
    D = torch.empty((128, 256), dtype=torch.float32, device=A.device)
    st = torch.zeros(1, dtype=torch.int32, device=A.device)
    _raise(lib().pxst_tensor_check(int(form), K, a, b, C.c_void_p(D.data_ptr()), C.c_void_p(st.data_ptr()),
                                   _stream(stream)), "tensor_check")
    return D, int(st.item())


def _scan_struct(rec):
    """pxst_scan for a Reconstruction's device-resident state."""
    p = lambda t: C.c_void_p(t.data_ptr())
    return _Scan(rec.dims.c(), rec.opts.c(), p(rec.frames), p(rec.W), p(rec.M), p(rec.delta), p(rec.u),
                 p(rec.I_ref), p(rec.w), p(rec.err), p(rec.ws), rec.ws.numel())


def autotune(rec, trials=3, stream=None):
    """pxst_autotune on a Reconstruction: (best tile, its median update time in ms). The
    scan's map is restored; rec.opts.tile is set to the choice."""
    sc = _scan_struct(rec)
    tile, ms = C.c_int32(0), C.c_float(0.0)
    _raise(lib().pxst_autotune(C.byref(sc), int(trials), _stream(stream), C.byref(tile), C.byref(ms)),
           "autotune")
    rec.opts.tile = int(tile.value)
    return int(tile.value), float(ms.value)


class Batch:
    """Many scans (Reconstruction objects, each with its own device state) iterated by one
    CUDA graph launch: pxst_batch_plan / pxst_batch_run. The scans' arrays must stay alive
    and in place while the batch exists."""

    def __init__(self, recs, n_iter, n_branches=8, autotune=False, stream=None):
        self.recs = list(recs)
        arr = (_Scan * len(self.recs))(*[_scan_struct(r) for r in self.recs])
        h = C.c_void_p()
        _raise(lib().pxst_batch_plan(arr, len(self.recs), int(n_iter), int(n_branches), 1 if autotune else 0,
                                     _stream(stream), C.byref(h)), "batch_plan")
        self._h = h

    def run(self, stream=None):
        _raise(lib().pxst_batch_run(self._h, _stream(stream)), "batch_run")

    def branch(self, i):
        return int(lib().pxst_batch_branch(self._h, int(i)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pxst_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def calc_error(dims: Dims, frames, W, M, I_ref, w, u, delta, ws, pixel_err=None, frame_err=None, total=None,
               ref_err=None, stream=None):
    """pxst_calc_error (section "Calculate figures of merit"); the outputs that are given
    (CUDA tensors: pixel_err float32 [ny][nx], frame_err float64 [N], total float64 [1],
    ref_err float32 [Ry][Rx]) are filled."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    opt = lambda t, dt, shape, name: _check(t, dt, shape, name) if t is not None else None
    _raise(lib().pxst_calc_error(C.byref(dims.c()), _check(frames, torch.float32, (N, ny, nx), "frames"),
                                 _check(W, torch.float32, (ny, nx), "W"), _check(M, torch.uint8, (ny, nx), "M"),
                                 _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
                                 _check(w, torch.float32, (Ry, Rx), "w"), _check(u, torch.float64, (2, ny, nx), "u"),
                                 _check(delta, torch.float64, (N, 2), "delta"),
                                 opt(pixel_err, torch.float32, (ny, nx), "pixel_err"),
                                 opt(frame_err, torch.float64, (N,), "frame_err"),
                                 opt(total, torch.float64, (1,), "total"),
                                 opt(ref_err, torch.float32, (Ry, Rx), "ref_err"),
                                 C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)), "calc_error")


def update_translations(dims: Dims, twindow, frames, W, M, I_ref, w, u, delta, ws, frame_err=None,
                        quadratic=True, stream=None):
    """pxst_update_translations (section "Update translations"): delta (float64 [N][2], CUDA)
    is updated in place; frame_err (float64 [N]) receives each frame's error at its minimum."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    _raise(lib().pxst_update_translations(C.byref(dims.c()), int(twindow[0]), int(twindow[1]),
                                          1 if quadratic else 0,
                                          _check(frames, torch.float32, (N, ny, nx), "frames"),
                                          _check(W, torch.float32, (ny, nx), "W"),
                                          _check(M, torch.uint8, (ny, nx), "M"),
                                          _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
                                          _check(w, torch.float32, (Ry, Rx), "w"),
                                          _check(u, torch.float64, (2, ny, nx), "u"),
                                          _check(delta, torch.float64, (N, 2), "delta"),
                                          _check(frame_err, torch.float64, (N,), "frame_err")
                                          if frame_err is not None else None,
                                          C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "update_translations")


def integrate_map(dims: Dims, M, u, ws, max_iter=100000, tol=1e-12, timeout_ns=0, stream=None):
    """pxst_integrate_map: the "integrate" option -- u (float64 [2][ny][nx], CUDA) made
    irrotational in place by least-squares integration and re-differentiation. Returns a CUDA
    float64 tensor [2]: the conjugate-gradient steps taken and the final relative residual."""
    torch = _torch()
    info = torch.zeros(2, dtype=torch.float64, device=u.device)
    _raise(lib().pxst_integrate_map(C.byref(dims.c()), _check(M, torch.uint8, (dims.ny, dims.nx), "M"),
                                    _check(u, torch.float64, (2, dims.ny, dims.nx), "u"), int(max_iter), float(tol),
                                    int(timeout_ns), C.c_void_p(info.data_ptr()), C.c_void_p(ws.data_ptr()),
                                    ws.numel(), _stream(stream)), "integrate_map")
    return info


def filter_map(dims: Dims, sigma, M, u, ws, stream=None):
    """pxst_filter_map: the "sigma" regularisation of the pixel map u (float64 [2][ny][nx],
    CUDA, in place)."""
    torch = _torch()
    _raise(lib().pxst_filter_map(C.byref(dims.c()), float(sigma), _check(M, torch.uint8, (dims.ny, dims.nx), "M"),
                                 _check(u, torch.float64, (2, dims.ny, dims.nx), "u"), C.c_void_p(ws.data_ptr()),
                                 ws.numel(), _stream(stream)), "filter_map")


def update_pixel_map_fractional(dims: Dims, opts: Options, sub, frames, W, M, I_ref, w, delta, u, ws, err=None,
                                stream=None):
    """pxst_update_pixel_map_fractional: the integer search, then candidates on a 1/sub grid
    within one pixel of its minimum (u updated in place)."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    _raise(lib().pxst_update_pixel_map_fractional(
        C.byref(dims.c()), C.byref(opts.c()), int(sub), _check(frames, torch.float32, (N, ny, nx), "frames"),
        _check(W, torch.float32, (ny, nx), "W"), _check(M, torch.uint8, (ny, nx), "M"),
        _check(I_ref, torch.float32, (Ry, Rx), "I_ref"), _check(w, torch.float32, (Ry, Rx), "w"),
        _check(delta, torch.float64, (N, 2), "delta"), _check(u, torch.float64, (2, ny, nx), "u"),
        _check(err, torch.float32, (ny, nx), "err") if err is not None else None,
        C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)), "update_pixel_map_fractional")


def defocus_sweep(dims: Dims, frames, W, M, u, delta, sy, sx, I_ref, w, ws, stream=None):
    """pxst_defocus_sweep: contrast of the reference image for every pair of map scales
    (sy[ky], sx[kx]) about the detector centre; returns a float64 CUDA tensor [len(sy)][len(sx)]."""
    torch = _torch()
    N, ny, nx, Ry, Rx = dims.n_frames, dims.ny, dims.nx, dims.ref_ny, dims.ref_nx
    sy = np.ascontiguousarray(sy, dtype=np.float64)
    sx = np.ascontiguousarray(sx, dtype=np.float64)
    out = torch.empty((sy.size, sx.size), dtype=torch.float64, device=frames.device)
    _raise(lib().pxst_defocus_sweep(C.byref(dims.c()), _check(frames, torch.float32, (N, ny, nx), "frames"),
                                    _check(W, torch.float32, (ny, nx), "W"), _check(M, torch.uint8, (ny, nx), "M"),
                                    _check(u, torch.float64, (2, ny, nx), "u"),
                                    _check(delta, torch.float64, (N, 2), "delta"),
                                    int(sy.size), sy.ctypes.data_as(C.c_void_p), int(sx.size),
                                    sx.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                                    _check(I_ref, torch.float32, (Ry, Rx), "I_ref"),
                                    _check(w, torch.float32, (Ry, Rx), "w"), C.c_void_p(ws.data_ptr()), ws.numel(),
                                    _stream(stream)), "defocus_sweep")
    return out
