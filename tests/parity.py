"""Parity criteria between the CUDA path and the FP64 oracle.

  * integer argmin: identical on >= 99.9 % of the pixels with M = 1; every other pixel must
    be a near-tie: the oracle's own error at the GPU's pick is within
    1e-5 * e_min + 1e-7 * (sum_n I^2 / var) of the oracle's minimum;
  * sub-pixel u: within 1e-3 px wherever the integer picks agree;
  * normalised error at the pick: relative 1e-4 (FP32 sums of at most a few hundred positive
    terms, each rounded at 2^-24, stay well inside it), plus an absolute floor for a pick whose
    residuals I - W R nearly vanish: a bilinear read in FP32 carries an absolute rounding of a
    few ulp of W R ~ I, so each squared residual is only known to about (2^-21 max_n |I_n|)^2,
    i.e. the error to N (2^-21 max_n |I_n|)^2 / var;
  * I_ref: relative L2 <= 1e-5 over reference pixels whose oracle weight exceeds
    1e-4 * max w (a few barely-covered edge pixels would otherwise dominate).
"""
from __future__ import annotations

import numpy as np

import oracle

ARGMIN_AGREE = 0.999
U_TOL = 1e-3
ERR_RTOL = 1e-4
IREF_RL2 = 1e-5


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2)) / max(np.sqrt(np.sum(b ** 2)), 1e-300))


def check_omap(Iref_gpu, w_gpu, Iref_or, w_or):
    sel = w_or > 1e-4 * w_or.max()
    r_i = rel_l2(Iref_gpu.astype(np.float64)[sel], Iref_or[sel])
    r_w = rel_l2(w_gpu.astype(np.float64), w_or)
    cov_mismatch = int(np.count_nonzero((w_gpu > 0) != (w_or > 0)))
    assert r_i <= IREF_RL2, f"I_ref relative L2 {r_i:.3e}"
    assert r_w <= IREF_RL2, f"w relative L2 {r_w:.3e}"
    # coverage may differ only where the weight is zero up to rounding
    assert cov_mismatch <= max(2, int(1e-4 * w_or.size)), cov_mismatch
    return dict(iref_rel_l2=r_i, w_rel_l2=r_w, coverage_mismatch=cov_mismatch)


def check_update(inp, pix, u_gpu_int, err_gpu_int, u_gpu_q, err_gpu_q, check_fit=True):
    """inp: dict(frames, W, M, Iref, w, delta, u, window) -- the oracle's inputs (Iref/w as
    used by both sides); pix: flat pixel indices to compare (all M = 1 pixels, or a sample);
    u_gpu_*: [2][K] for those pixels; err_gpu_*: [K]. check_fit=False checks the integer
    picks and their errors only."""
    frames, W, M, Iref, w, delta, u, window = (inp[k] for k in
                                               ("frames", "W", "M", "Iref", "w", "delta", "u", "window"))
    pix = np.asarray(pix, dtype=np.int64)
    uo_int, eo_int = oracle.update_pixels(frames, W, M, Iref, w, delta, u, window, pix, quadratic=False)
    if check_fit:
        uo_q, eo_q = oracle.update_pixels(frames, W, M, Iref, w, delta, u, window, pix, quadratic=True)
    else:
        uo_q, u_gpu_q = uo_int, u_gpu_int
    uo_int, uo_q = uo_int.T, uo_q.T
    same = np.all(u_gpu_int == uo_int, axis=0)
    agree = float(np.mean(same)) if pix.size else 1.0
    bad = np.nonzero(~same)[0]
    ny, nx = M.shape
    Sy, Sx = window
    worst_gap = 0.0
    for k in bad:
        p = int(pix[k])
        e, (ci, cj) = oracle.pixel_window(frames, W, M, Iref, w, delta, u, window, p)
        a = int(round(u_gpu_int[0, k])) - ci + Sy
        b = int(round(u_gpu_int[1, k])) - cj + Sx
        assert 0 <= a <= 2 * Sy and 0 <= b <= 2 * Sx, (p, a, b)
        I = frames[:, p // nx, p % nx].astype(np.float64)
        Wv = float(W.ravel()[p])
        scale = float(np.sum(I * I) / max(np.sum((I - Wv) ** 2), 1e-300))
        emin = float(np.min(e))
        gap = float(e[a, b] - emin)
        tol = 1e-5 * emin + 1e-7 * scale
        assert gap <= tol, f"pixel {p}: GPU pick is {gap:.3e} above the minimum (tolerance {tol:.3e})"
        worst_gap = max(worst_gap, gap / max(tol, 1e-300))
    assert agree >= ARGMIN_AGREE, f"integer argmin agreement {agree:.5f}"
    # sub-pixel map where the integer picks agree
    du = np.abs(u_gpu_q - uo_q)[:, same]
    max_du = float(du.max()) if du.size else 0.0
    assert max_du <= U_TOL, f"sub-pixel u differs by {max_du:.3e} px"
    fin = same & np.isfinite(eo_int)
    # the absolute floor of the error at the pick (module docstring), per pixel
    fr = frames.reshape(frames.shape[0], -1)[:, pix].astype(np.float64)
    Wp = W.ravel()[pix].astype(np.float64)
    var_all = np.maximum(np.sum((fr - Wp) ** 2, axis=0), 1e-300)
    floor = fr.shape[0] * (2.0 ** -21 * np.max(np.abs(fr), axis=0)) ** 2 / var_all
    dev = np.abs(err_gpu_int[fin] - eo_int[fin])
    rel = np.maximum(dev - floor[fin], 0.0) / np.maximum(np.abs(eo_int[fin]), 1e-30)
    max_rel = float(rel.max()) if rel.size else 0.0
    assert max_rel <= ERR_RTOL, f"error at the pick differs by {max_rel:.3e} (relative, beyond the rounding floor)"
    # non-finite errors (no valid candidate) must match exactly
    assert np.array_equal(np.isinf(err_gpu_int[same]), np.isinf(eo_int[same]))
    return dict(pixels=int(pix.size), argmin_agree=agree, near_ties=int(bad.size),
                max_du=max_du, rms_du=float(np.sqrt(np.mean(du ** 2))) if du.size else 0.0,
                max_err_rel=max_rel, worst_tie_ratio=worst_gap)


def check_iteration(s, u_start, gpu_int, gpu_q):
    """One main-loop iteration on the GPU against the oracle, with the full criterion.

    gpu_int, gpu_q: (u, err, I_ref, w) of the GPU's iteration from u_start without and with
    the 3x3 fit. The GPU's reference image must match the oracle's make_object_map from
    u_start (check_omap); the GPU's update must then pass check_update against the oracle's
    update run on the GPU's own reference image and weights read back as FP64, so that both
    sides search the same reference and every differing pick must be an oracle near-tie."""
    u_i, e_i, I_i, w_i = gpu_int
    u_q, e_q, I_q, w_q = gpu_q
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, u_start, s.delta, s.ref_shape)
    rep_o = check_omap(I_q, w_q, Io, wo)
    # both calls build their reference from the same map: identical up to the FP64 atomics' order
    assert rel_l2(I_i.astype(np.float64), I_q.astype(np.float64)) < 1e-6
    inp = dict(frames=s.frames, W=s.W, M=s.M, Iref=I_q.astype(np.float64), w=w_q.astype(np.float64),
               delta=s.delta, u=u_start, window=s.window)
    if not np.array_equal(I_i, I_q):
        # the integer call searched its own (rounding-level different) reference: rerun
        # the comparison of its picks against that one
        inp_i = dict(inp, Iref=I_i.astype(np.float64), w=w_i.astype(np.float64))
    else:
        inp_i = inp
    pix = np.flatnonzero(s.M.ravel())
    rep_u = check_update(inp, pix, u_i.reshape(2, -1)[:, pix], e_i.ravel()[pix], u_q.reshape(2, -1)[:, pix],
                         e_q.ravel()[pix]) if inp_i is inp else _check_split(inp_i, inp, pix, u_i, e_i, u_q, e_q)
    return dict(omap=rep_o, update=rep_u)


def _check_split(inp_i, inp_q, pix, u_i, e_i, u_q, e_q):
    """check_update when the integer and fitted GPU calls searched references that differ by
    rounding: the integer picks against the oracle on the first, the fit on the second
    (where the integer picks of both calls agree)."""
    rep = check_update(inp_i, pix, u_i.reshape(2, -1)[:, pix], e_i.ravel()[pix], u_i.reshape(2, -1)[:, pix],
                       e_i.ravel()[pix], check_fit=False)
    uo_i, _ = oracle.update_pixels(inp_q["frames"], inp_q["W"], inp_q["M"], inp_q["Iref"], inp_q["w"],
                                   inp_q["delta"], inp_q["u"], inp_q["window"], pix, quadratic=False)
    uo_q, _ = oracle.update_pixels(inp_q["frames"], inp_q["W"], inp_q["M"], inp_q["Iref"], inp_q["w"],
                                   inp_q["delta"], inp_q["u"], inp_q["window"], pix, quadratic=True)
    same = np.all(u_i.reshape(2, -1)[:, pix] == uo_i.T, axis=0)
    du = np.abs(u_q.reshape(2, -1)[:, pix] - uo_q.T)[:, same]
    max_du = float(du.max()) if du.size else 0.0
    assert max_du <= U_TOL, f"sub-pixel u differs by {max_du:.3e} px"
    rep["max_du"] = max_du
    return rep
