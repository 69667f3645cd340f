"""Seeded synthetic PXST scans: the inputs that both the oracle and the CUDA path consume.

This module renders measured frames from the paper's forward model (Eq. 1, and its
discrete form in the "Initialisation" section): I[n,i,j] = W[i,j] * I_ref(u[i,j] - Delta[n]).
It holds none of the reconstruction arithmetic (no make_object_map, no pixel-map search,
no bilinear interpolation): the reference image here is a *continuous* field,
I_ref(p) = sum_m a_m g(p - m), a sum of truncated Gaussians centred on integer grid
points with uniform random amplitudes a_m, evaluated exactly wherever a frame samples it.
A bilinear interpolant of the grid would bias the truth-recovery pins toward the method's
own interpolation, so it is deliberately not used.

Most pixel maps generated here are separable, u[0] = fy(i) and u[1] = fx(j), which makes
the rendering a pair of 1-D band sums per frame; `make_scan_general` renders any map (a
rotation or a curl term couples the axes) by evaluating the field at every sample point,
and can mark isolated bad pixels inside the good region of the mask.

Conventions (shared with the C ABI):
  frames  float32 [N][ny][nx]      Poisson counts (or the noiseless expectation)
  W       float32 [ny][nx]         whitefield
  M       uint8   [ny][nx]         1 = good pixel (W >= 5 % of its peak)
  u       float64 [2][ny][nx]      u[0] slow-scan (row) and u[1] fast-scan (column),
                                   in reference-pixel units
  delta   float64 [N][2]           (Delta_i[n], Delta_j[n]) in reference-pixel units
  Iref_true float64 [Ry][Rx]       the continuous field sampled at integer points
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 12726


@dataclass
class Scan:
    name: str
    frames: np.ndarray
    W: np.ndarray
    M: np.ndarray
    u_true: np.ndarray
    u_init: np.ndarray
    delta: np.ndarray
    ref_shape: tuple
    Iref_true: np.ndarray
    window: tuple          # (S_y, S_x): candidates span [-S, S] on each axis
    n_iter: int
    sigma: float
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        n, ny, nx = self.frames.shape
        return (n, ny, nx, self.ref_shape[0], self.ref_shape[1])


# --------------------------------------------------------------------------------------
# continuous reference field
# --------------------------------------------------------------------------------------

def _kernel(d, sigma):
    """Gaussian of width sigma, truncated at 4 sigma and lowered so it reaches 0 there."""
    r = 4.0 * sigma
    return np.where(np.abs(d) < r, np.exp(-d * d / (2.0 * sigma * sigma)) - np.exp(-8.0), 0.0)


class Field:
    """I(p) = 0.5 + (sum_m a_m g(p_y - m_y) g(p_x - m_x) - lo) / (hi - lo).

    a_m ~ U[0, 1) on integer points covering the reference grid plus a margin;
    lo/hi are the min/max of the raw sum over the reference grid's integer points,
    so the grid samples span exactly [0.5, 1.5].
    """

    def __init__(self, ref_shape, sigma, rng):
        self.sigma = float(sigma)
        self.K = int(np.ceil(4.0 * sigma)) + 1
        self.pad = self.K + 2
        Ry, Rx = ref_shape
        self.a = rng.random((Ry + 2 * self.pad, Rx + 2 * self.pad))
        self.lo, self.hi = 0.0, 1.0
        grid = self._raw(np.arange(Ry, dtype=np.float64), np.arange(Rx, dtype=np.float64))
        self.lo, self.hi = float(grid.min()), float(grid.max())

    def _taps(self, p):
        base = np.floor(p).astype(np.int64)
        offs = np.arange(-self.K, self.K + 1)
        m = base[:, None] + offs[None, :]
        w = _kernel(p[:, None] - m, self.sigma)
        idx = m + self.pad
        if idx.min() < 0 or idx.max() >= max(self.a.shape):
            raise ValueError("field evaluated too far outside its coefficient grid")
        return idx, w

    def _raw(self, py, px):
        iy, wy = self._taps(py)
        ix, wx = self._taps(px)
        if iy.max() >= self.a.shape[0] or ix.max() >= self.a.shape[1]:
            raise ValueError("field evaluated too far outside its coefficient grid")
        r0, r1 = int(iy.min()), int(iy.max()) + 1
        rows = self.a[r0:r1]
        t = np.zeros((r1 - r0, px.size))
        for k in range(ix.shape[1]):
            t += rows[:, ix[:, k]] * wx[:, k][None, :]
        out = np.zeros((py.size, px.size))
        for k in range(iy.shape[1]):
            out += t[iy[:, k] - r0, :] * wy[:, k][:, None]
        return out

    def separable(self, py, px):
        """Field on the outer product of row positions py and column positions px."""
        return 0.5 + (self._raw(np.asarray(py, np.float64), np.asarray(px, np.float64)) - self.lo) / (self.hi - self.lo)

    def points(self, py, px, chunk=1 << 14):
        """Field at arbitrary points (py[k], px[k]): every point sums its (2K+1)^2 taps,
        in chunks of points evaluated on a thread pool."""
        py = np.ascontiguousarray(py, np.float64).ravel()
        px = np.ascontiguousarray(px, np.float64).ravel()
        out = np.empty(py.size)

        def one(k0):
            k1 = min(py.size, k0 + chunk)
            iy, wy = self._taps(py[k0:k1])
            ix, wx = self._taps(px[k0:k1])
            if iy.max() >= self.a.shape[0] or ix.max() >= self.a.shape[1]:
                raise ValueError("field evaluated too far outside its coefficient grid")
            # sum over the row taps of (row tap weight x the row's column-tap sum)
            flat = self.a.ravel()
            acc = np.zeros(k1 - k0)
            for r in range(iy.shape[1]):
                taps = flat[iy[:, r, None] * self.a.shape[1] + ix]       # [points][2K+1]
                acc += wy[:, r] * np.einsum("kj,kj->k", taps, wx)
            out[k0:k1] = acc
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(one, range(0, py.size, chunk)))
        return 0.5 + (out - self.lo) / (self.hi - self.lo)

    def grid(self, ref_shape):
        Ry, Rx = ref_shape
        return self.separable(np.arange(Ry, dtype=np.float64), np.arange(Rx, dtype=np.float64))


# --------------------------------------------------------------------------------------
# generic separable scan
# --------------------------------------------------------------------------------------

def _threads():
    return max(1, min(16, os.cpu_count() or 1))


def make_scan(name, *, ny, nx, ref_shape, sigma, delta, uy, ux, uy0, ux0, W, window, n_iter,
              seed, noise=True, extra=None):
    """Render a scan whose pixel map is separable: u[0][i,j] = uy[i], u[1][i,j] = ux[j].

    uy/ux are the true maps, uy0/ux0 the initial estimate; W is [ny][nx].
    """
    rng = np.random.default_rng(seed)
    fld = Field(ref_shape, sigma, rng)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    n = delta.shape[0]
    frames = np.empty((n, ny, nx), dtype=np.float32)
    Wd = np.asarray(W, dtype=np.float64)

    def render(k):
        f = fld.separable(uy - delta[k, 0], ux - delta[k, 1])
        return k, Wd * f

    expect = np.empty((n, ny, nx), dtype=np.float64) if noise else None
    with ThreadPoolExecutor(_threads()) as ex:
        for k, img in ex.map(render, range(n)):
            if noise:
                expect[k] = img
            else:
                frames[k] = img.astype(np.float32)
    if noise:
        # Poisson counts drawn in frame order from the scan's own generator
        for k in range(n):
            frames[k] = rng.poisson(expect[k]).astype(np.float32)
        del expect

    u_true = np.empty((2, ny, nx), dtype=np.float64)
    u_true[0] = np.asarray(uy, np.float64)[:, None]
    u_true[1] = np.asarray(ux, np.float64)[None, :]
    u_init = np.empty_like(u_true)
    u_init[0] = np.asarray(uy0, np.float64)[:, None]
    u_init[1] = np.asarray(ux0, np.float64)[None, :]
    Wf = np.ascontiguousarray(Wd.astype(np.float32))
    M = (Wd >= 0.05 * Wd.max()).astype(np.uint8)
    return Scan(name=name, frames=frames, W=Wf, M=M, u_true=u_true, u_init=u_init,
                delta=delta, ref_shape=tuple(int(v) for v in ref_shape),
                Iref_true=fld.grid(ref_shape), window=tuple(window), n_iter=n_iter,
                sigma=sigma, meta=dict(seed=seed, noise=noise, **(extra or {})))


def make_scan_general(name, *, ref_shape, sigma, delta, u_true, u_init, W, window, n_iter, seed, noise=True,
                      bad_frac=0.0, extra=None):
    """Render a scan with any pixel map u_true [2][ny][nx] (u_init: the initial estimate):
    frame n samples the continuous field at u_true - Delta[n] point by point. With
    bad_frac > 0 that fraction of the good pixels (W >= 5 % of its peak), drawn at random
    among those whose 8 neighbours are all good, is marked bad (M = 0): isolated defects
    inside the good region, as a mask made from outliers against their neighbours has."""
    rng = np.random.default_rng(seed)
    fld = Field(ref_shape, sigma, rng)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    u_true = np.ascontiguousarray(u_true, dtype=np.float64)
    n = delta.shape[0]
    _, ny, nx = u_true.shape
    Wd = np.asarray(W, dtype=np.float64)
    frames = np.empty((n, ny, nx), dtype=np.float32)
    for k in range(n):
        f = fld.points(u_true[0] - delta[k, 0], u_true[1] - delta[k, 1]).reshape(ny, nx)
        img = Wd * f
        frames[k] = (rng.poisson(img) if noise else img).astype(np.float32)
    M = (Wd >= 0.05 * Wd.max()).astype(np.uint8)
    if bad_frac > 0:
        inner = np.zeros_like(M)
        good = M > 0
        inner[1:-1, 1:-1] = good[1:-1, 1:-1] & good[:-2, 1:-1] & good[2:, 1:-1] & good[1:-1, :-2] & \
            good[1:-1, 2:] & good[:-2, :-2] & good[:-2, 2:] & good[2:, :-2] & good[2:, 2:]
        cand = np.flatnonzero(inner.ravel())
        k = int(round(bad_frac * good.sum()))
        # isolated: a drawn pixel none of whose 8 neighbours was drawn before it
        chosen = np.zeros(M.size, dtype=bool)
        for p in rng.permutation(cand):
            if k == 0:
                break
            i, j = divmod(int(p), nx)
            if not chosen.reshape(ny, nx)[i - 1:i + 2, j - 1:j + 2].any():
                chosen[p] = True
                k -= 1
        M.ravel()[chosen] = 0
    return Scan(name=name, frames=frames, W=np.ascontiguousarray(Wd.astype(np.float32)), M=M, u_true=u_true,
                u_init=np.ascontiguousarray(u_init, dtype=np.float64), delta=delta,
                ref_shape=tuple(int(v) for v in ref_shape), Iref_true=fld.grid(ref_shape), window=tuple(window),
                n_iter=n_iter, sigma=sigma, meta=dict(seed=seed, noise=noise, bad_frac=bad_frac, **(extra or {})))


def nonsep2d(n_side=4, det=64, step=6, ref=170, sigma=2.0, mag=1.3, offset=40.0, theta=0.03, curl=0.8,
             aberr=2.0, window=5, n_iter=3, seed=BASE_SEED + 30, noise=True, bad_frac=0.01, ny=None, nx=None,
             peak=1000.0, w_sigma=None, jitter=0.0, name=None):
    """A 2-D scan whose pixel map couples the axes: a small rotation theta (curl 2 theta)
    and a sinusoidal shear of amplitude `curl` on top of the magnification and a cubic
    aberration per axis,
        u_y = offset + mag y - theta (x - cx) + aberr t_y^3 + curl sin(2 pi x / nx),
        u_x = offset + mag x + theta (y - cy) + aberr t_x^3 + curl sin(2 pi y / ny),
    so a tile's candidate windows do not stack into rows and columns; the initial map is the
    linear part (no aberration, no shear). Translations on an n_side^2 grid of `step`
    (plus a uniform jitter of up to `jitter` px per axis, from its own seeded stream: a
    fractional part on both axes), Gaussian whitefield, and bad_frac of the good pixels
    marked bad at random."""
    ny = det if ny is None else ny
    nx = det if nx is None else nx
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    cy, cx = (ny - 1) / 2.0, (nx - 1) / 2.0
    ty, tx = (y - cy) / max(cy, 1.0), (x - cx) / max(cx, 1.0)
    lin_y = offset + mag * y - theta * (x - cx)
    lin_x = offset + mag * x + theta * (y - cy)
    u_true = np.stack(np.broadcast_arrays(lin_y + aberr * ty ** 3 + curl * np.sin(2 * np.pi * x / nx),
                                          lin_x + aberr * tx ** 3 + curl * np.sin(2 * np.pi * y / ny)))
    u_init = np.stack(np.broadcast_arrays(lin_y + 0.0 * x, lin_x + 0.0 * y))
    ws = w_sigma if w_sigma is not None else 0.34 * max(ny, nx)
    W = peak * np.exp(-((y - cy) ** 2 + (x - cx) ** 2) / (2.0 * ws * ws))
    rs = (ref, ref) if np.isscalar(ref) else tuple(ref)
    delta = grid_delta(n_side, step)
    if jitter > 0:
        delta = delta + np.random.default_rng(seed + 1).uniform(0.0, jitter, size=delta.shape)
    return make_scan_general(name or f"nonsep2d-{n_side * n_side}x{ny}x{nx}-w{window}", ref_shape=rs, sigma=sigma,
                             delta=delta, u_true=u_true, u_init=u_init, W=W,
                             window=(window, window), n_iter=n_iter, seed=seed, noise=noise, bad_frac=bad_frac,
                             extra=dict(theta=theta, curl=curl))


# --------------------------------------------------------------------------------------
# the workloads (sizes after the paper's example data set, 121 frames of 516 x 1556,
# and the 2-D scans it describes)
# --------------------------------------------------------------------------------------

def grid_delta(n_side, step):
    """Translations on an n_side x n_side grid, row-major, (Delta_i, Delta_j) = step*(a, b)."""
    a, b = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    return np.stack([step * a.ravel(), step * b.ravel()], axis=1).astype(np.float64)


def tiny2d(n_side=4, det=64, step=6, ref=160, sigma=2.0, mag=1.5, offset=30.0, aberr=3.0,
           window=4, n_iter=5, seed=BASE_SEED, noise=True, peak=1000.0, w_sigma=None, name=None):
    """2-D scan after the small configuration: n_side^2 frames of det x det pixels,
    u = offset + mag*x + aberr*t^3 with t = (x - c)/c on each axis, Gaussian whitefield."""
    x = np.arange(det, dtype=np.float64)
    c = (det - 1) / 2.0
    t = (x - c) / max(c, 1.0)
    u = offset + mag * x + aberr * t ** 3
    u0 = offset + mag * x
    ws = w_sigma if w_sigma is not None else 22.0 * det / 64.0
    yy, xx = np.meshgrid(x - c, x - c, indexing="ij")
    W = peak * np.exp(-(yy ** 2 + xx ** 2) / (2.0 * ws * ws))
    return make_scan(name or f"2d-{n_side * n_side}x{det}x{det}", ny=det, nx=det,
                     ref_shape=(ref, ref), sigma=sigma, delta=grid_delta(n_side, step),
                     uy=u, ux=u, uy0=u0, ux0=u0, W=W, window=(window, window),
                     n_iter=n_iter, seed=seed, noise=noise)


def config_small(noise=True):
    """16 frames of 64 x 64, 4x4 grid of 6 px steps, reference 160 x 160, sigma 2,
    u = 30 + 1.5 x + 3 t^3, window +-4, 5 iterations."""
    return tiny2d(noise=noise, seed=BASE_SEED + 0, name="2d-16x64x64-w4")


def config_lens1d(noise=True, n_frames=121, ny=512, nx=1536, step=0.8, seed=BASE_SEED + 1):
    """1-D lens-like scan: 121 frames of 512 x 1536, translations along the fast axis only
    in 0.8 px steps; u_fs = o + x (1 + 0.1 x / (nx-1)) + 20 t^5, u_ss = ss + 4;
    whitefield = Gaussian (sigma 400 px) along fs times a smoothed top-hat along ss;
    window +-1 (ss) x +-24 (fs), 10 iterations."""
    fs = np.arange(nx, dtype=np.float64)
    ss = np.arange(ny, dtype=np.float64)
    o = 128.0
    c = (nx - 1) / 2.0
    t = (fs - c) / c
    ux0 = o + fs * (1.0 + 0.1 * fs / (nx - 1))
    ux = ux0 + 20.0 * t ** 5
    uy = ss + 4.0
    span = step * (n_frames - 1)
    ref = (ny + 8, int(np.ceil(o + (nx - 1) * 1.1 + 20.0 + 72.0)))
    delta = np.stack([np.zeros(n_frames), step * np.arange(n_frames)], axis=1)
    # the reference must hold u - Delta for every frame
    lo = ux0.min() - 20.0 - span
    if lo < 8:
        raise ValueError("reference offset too small for the scan span")
    gx = np.exp(-((fs - c) ** 2) / (2.0 * 400.0 ** 2))
    edge = 2.0
    th = 1.0 / (1.0 + np.exp(-(ss - 16.0) / edge)) / (1.0 + np.exp((ss - (ny - 16.0)) / edge))
    W = 1000.0 * th[:, None] * gx[None, :]
    return make_scan(f"1d-{n_frames}x{ny}x{nx}-w1x24", ny=ny, nx=nx, ref_shape=ref, sigma=2.0,
                     delta=delta, uy=uy, ux=ux, uy0=uy, ux0=ux0, W=W, window=(1, 24),
                     n_iter=10, seed=seed, noise=noise)


def config_precision2d(noise=True, n_side=20, det=1024, step=4, ref=1200, seed=BASE_SEED + 2):
    """400 frames (20 x 20 grid, 4 px step) of 1024 x 1024, reference 1200 x 1200, speckle
    sigma 1.5; u = 104 + 1.02 x + 8 t^3 on each axis; window +-16 x +-16."""
    x = np.arange(det, dtype=np.float64)
    c = (det - 1) / 2.0
    t = (x - c) / c
    u0 = 104.0 + 1.02 * x
    u = u0 + 8.0 * t ** 3
    yy, xx = np.meshgrid(x - c, x - c, indexing="ij")
    W = 1000.0 * np.exp(-(yy ** 2 + xx ** 2) / (2.0 * 400.0 ** 2))
    return make_scan(f"2d-{n_side * n_side}x{det}x{det}-w16", ny=det, nx=det, ref_shape=(ref, ref),
                     sigma=1.5, delta=grid_delta(n_side, step), uy=u, ux=u, uy0=u0, ux0=u0, W=W,
                     window=(16, 16), n_iter=10, seed=seed, noise=noise)


CONFIGS = {
    "small": config_small,
    "lens1d": config_lens1d,
    "precision2d": config_precision2d,
}
