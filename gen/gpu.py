"""The same synthetic scans rendered on a GPU (torch), for the batched and served workloads,
whose dozens to hundreds of scans of up to 400 x 1024 x 1024 frames the host renderer
would take minutes to produce.

The reference field is the host generator's continuous field (a separable sum of
truncated Gaussians on integer points with uniform amplitudes, affinely mapped so that its
grid samples span [0.5, 1.5]); because every pixel map here is separable, a frame is
W * (G_y a G_x^T), with G_y[i, m] = g(u_y[i] - Delta_y - m) and G_x likewise, two dense
FP32 products. The random stream is torch's, seeded per scan, so a GPU-rendered scan is a
different draw than the host generator's scan of the same seed. Holds no reconstruction
arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class DeviceScan:
    name: str
    frames: "torch.Tensor"   # float32 [N][ny][nx]
    W: "torch.Tensor"        # float32 [ny][nx]
    M: "torch.Tensor"        # uint8 [ny][nx]
    delta: "torch.Tensor"    # float64 [N][2]
    u_init: "torch.Tensor"   # float64 [2][ny][nx]
    ref_shape: tuple
    window: tuple

    @property
    def dims(self):
        n, ny, nx = self.frames.shape
        return (int(n), int(ny), int(nx), int(self.ref_shape[0]), int(self.ref_shape[1]))

    @property
    def evals(self):
        Sy, Sx = self.window
        return int(self.M.sum().item()) * (2 * Sy + 1) * (2 * Sx + 1) * int(self.frames.shape[0])

    def nbytes(self):
        return sum(t.numel() * t.element_size() for t in (self.frames, self.W, self.M, self.delta, self.u_init))


class _Field:
    def __init__(self, ref_shape, sigma, g, device):
        import torch
        self.sigma = float(sigma)
        self.K = int(math.ceil(4.0 * sigma)) + 1
        self.pad = self.K + 2
        Ry, Rx = ref_shape
        self.a = torch.rand((Ry + 2 * self.pad, Rx + 2 * self.pad), generator=g, device=device,
                            dtype=torch.float32)
        self.lo, self.hi = 0.0, 1.0
        raw = self._raw(torch.arange(Ry, device=device, dtype=torch.float64),
                        torch.arange(Rx, device=device, dtype=torch.float64))
        self.lo, self.hi = float(raw.min()), float(raw.max())

    def _G(self, p, n):
        import torch
        m = torch.arange(n, device=p.device, dtype=torch.float64) - self.pad
        d = p[:, None] - m[None, :]
        r = 4.0 * self.sigma
        g = torch.exp(-d * d / (2.0 * self.sigma * self.sigma)) - math.exp(-8.0)
        return torch.where(d.abs() < r, g, torch.zeros_like(g)).to(torch.float32)

    def _raw(self, py, px):
        Gy = self._G(py, self.a.shape[0])
        Gx = self._G(px, self.a.shape[1])
        return (Gy @ self.a) @ Gx.T

    def separable(self, py, px):
        return 0.5 + (self._raw(py, px) - self.lo) / (self.hi - self.lo)


def _render(name, *, ny, nx, ref_shape, sigma, delta, uy, ux, uy0, ux0, W, window, seed, device, noise=True):
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False            # FP32 products
    try:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        fld = _Field(ref_shape, sigma, g, device)
        dl = torch.as_tensor(np.asarray(delta, np.float64), device=device)
        uyt = torch.as_tensor(np.asarray(uy, np.float64), device=device)
        uxt = torch.as_tensor(np.asarray(ux, np.float64), device=device)
        Wt = torch.as_tensor(np.asarray(W, np.float32), device=device)
        n = dl.shape[0]
        frames = torch.empty((n, ny, nx), dtype=torch.float32, device=device)
        for k in range(n):
            img = Wt * fld.separable(uyt - dl[k, 0], uxt - dl[k, 1])
            frames[k] = torch.poisson(img.clamp_min(0.0), generator=g) if noise else img
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    u0 = torch.empty((2, ny, nx), dtype=torch.float64, device=device)
    u0[0] = torch.as_tensor(np.asarray(uy0, np.float64), device=device)[:, None]
    u0[1] = torch.as_tensor(np.asarray(ux0, np.float64), device=device)[None, :]
    M = (Wt >= 0.05 * Wt.max()).to(torch.uint8)
    return DeviceScan(name, frames.contiguous(), Wt.contiguous(), M.contiguous(), dl.contiguous(), u0,
                      tuple(int(v) for v in ref_shape), tuple(int(v) for v in window))


def scan2d(n_side, det, window, *, step=6.0, sigma=2.0, mag=1.5, offset=30.0, aberr=3.0, seed, device="cuda",
           noise=True):
    """The small configuration's 2-D geometry at any size: n_side^2 frames on a grid of
    `step`, det x det pixels, u = offset + mag x + aberr t^3 per axis, Gaussian whitefield
    of width 22 det / 64 and peak 1000; the reference just covers every frame's footprint."""
    x = np.arange(det, dtype=np.float64)
    c = (det - 1) / 2.0
    t = (x - c) / max(c, 1.0)
    u = offset + mag * x + aberr * t ** 3
    u0 = offset + mag * x
    a, b = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    delta = np.stack([step * a.ravel(), step * b.ravel()], axis=1).astype(np.float64)
    ws = 22.0 * det / 64.0
    yy, xx = np.meshgrid(x - c, x - c, indexing="ij")
    W = 1000.0 * np.exp(-(yy ** 2 + xx ** 2) / (2.0 * ws * ws))
    R = int(math.ceil(u.max() + abs(aberr) + window + 8))
    return _render(f"2d-{n_side * n_side}x{det}x{det}-w{window}", ny=det, nx=det, ref_shape=(R, R), sigma=sigma,
                   delta=delta, uy=u, ux=u, uy0=u0, ux0=u0, W=W, window=(window, window), seed=seed, device=device,
                   noise=noise)


def scan1d(n_frames, ny, nx, *, step=0.8, sigma=2.0, seed, device="cuda", noise=True):
    """The 1-D lens geometry at any size: translations along the fast axis in `step`
    pixels, u_fs = o + x (1 + 0.1 x / (nx - 1)) + 20 t^5, u_ss = ss + 4, whitefield
    Gaussian along fs times a smoothed top-hat along ss, window +-1 x +-24."""
    fs = np.arange(nx, dtype=np.float64)
    ss = np.arange(ny, dtype=np.float64)
    o = 8.0 + step * (n_frames - 1)
    t = (fs - (nx - 1) / 2.0) / max((nx - 1) / 2.0, 1.0)
    ux = o + fs * (1.0 + 0.1 * fs / max(nx - 1, 1)) + 20.0 * t ** 5
    ux0 = o + fs * (1.0 + 0.1 * fs / max(nx - 1, 1))
    uy = ss + 4.0
    delta = np.zeros((n_frames, 2))
    delta[:, 1] = step * np.arange(n_frames)
    wfs = np.exp(-((fs - (nx - 1) / 2.0) ** 2) / (2.0 * (0.26 * nx) ** 2))
    e = max(ny * 0.04, 1.0)
    wss = 1.0 / (1.0 + np.exp(-(ss - 0.06 * ny) / e)) / (1.0 + np.exp((ss - 0.94 * ny) / e))
    W = 1000.0 * wss[:, None] * wfs[None, :]
    Ry = ny + 8 + 8
    Rx = int(math.ceil(ux.max() + 24 + 8))
    return _render(f"1d-{n_frames}x{ny}x{nx}-w1x24", ny=ny, nx=nx, ref_shape=(Ry, Rx), sigma=sigma, delta=delta,
                   uy=uy, ux=ux, uy0=uy, ux0=ux0, W=W, window=(1, 24), seed=seed, device=device, noise=noise)


def batch_specs(n_scans=64, seed=12726 + 3):
    """The batched workload: the small configuration's generator with frames ~U[16, 400]
    (a square grid of translations), detector sides ~U[128, 1024] and windows ~U{4..16}."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scans):
        frames = int(rng.integers(16, 401))
        out.append(dict(kind="2d", n_side=max(4, int(round(math.sqrt(frames)))), det=int(rng.integers(128, 1025)),
                        window=int(rng.integers(4, 17)), seed=seed * 1000 + k))
    return out


def serve_specs(n_scans=500, seed=12726 + 4):
    """The served workload: sizes log-uniform between the small configuration (16 frames of
    64 x 64) and the 2-D precision scan (400 frames of 1024 x 1024), 1-D or 2-D geometry with
    probability 1/2 each."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scans):
        tau = float(rng.random())
        frames = int(round(16 * 25 ** tau))
        side = int(round(64 * 16 ** tau))
        if rng.random() < 0.5:
            out.append(dict(kind="2d", n_side=max(4, int(round(math.sqrt(frames)))), det=side,
                            window=int(round(4 + 12 * tau)), seed=seed * 1000 + k))
        else:
            out.append(dict(kind="1d", n_frames=frames, ny=max(16, side // 2), nx=max(96, (3 * side) // 2),
                            seed=seed * 1000 + k))
    return out


def render(spec, device="cuda"):
    if spec["kind"] == "2d":
        return scan2d(spec["n_side"], spec["det"], spec["window"], seed=spec["seed"], device=device)
    return scan1d(spec["n_frames"], spec["ny"], spec["nx"], seed=spec["seed"], device=device)


def spec_dims(spec):
    """(N, ny, nx, Ry, Rx) and window of a spec without rendering it."""
    if spec["kind"] == "2d":
        det, ns, wnd = spec["det"], spec["n_side"], spec["window"]
        x = np.arange(det, dtype=np.float64)
        c = (det - 1) / 2.0
        t = (x - c) / max(c, 1.0)
        u = 30.0 + 1.5 * x + 3.0 * t ** 3
        R = int(math.ceil(u.max() + 3.0 + wnd + 8))
        return (ns * ns, det, det, R, R), (wnd, wnd)
    n, ny, nx = spec["n_frames"], spec["ny"], spec["nx"]
    fs = np.arange(nx, dtype=np.float64)
    o = 8.0 + 0.8 * (n - 1)
    t = (fs - (nx - 1) / 2.0) / max((nx - 1) / 2.0, 1.0)
    ux = o + fs * (1.0 + 0.1 * fs / max(nx - 1, 1)) + 20.0 * t ** 5
    return (n, ny, nx, ny + 16, int(math.ceil(ux.max() + 24 + 8))), (1, 24)
