"""Pins for the FP64 oracle: checks against what the paper and the mathematics fix.

Each ``pin_*`` takes an oracle library handle ``L`` (the real build, or a build of a copy
of the source with a planted mistake) and raises AssertionError if the oracle disagrees
with a value or property that does not come from the oracle itself:

  * worked values of the paper's bilinear formulas (tests/golden/*.txt),
  * closed forms (bilinear interpolation reproduces a + b x + c y + d x y exactly; a least
    squares paraboloid through an exact paraboloid returns its vertex; a quadratic error
    surface has its minimum at the true shift),
  * invariants (conservation of the scattered weight and of its first moment, a
    constant reference is returned unchanged),
  * exact special cases (integer maps reproduce the reference exactly; noiseless data
    with integer truth has zero error at the truth),
  * the same error computed a second way (plain array indexing for integer shifts),
  * statistical truth recovery on noiseless data (0.01 px RMS at 400 frames).
"""
from __future__ import annotations

import os

import numpy as np

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(line.split())
    return out


# ---------------------------------------------------------------------------------------
# bilinear interpolation and assignment (section "Sub-pixel interpolation")
# ---------------------------------------------------------------------------------------

def pin_bilinear_golden(L):
    for r in _rows("bilinear_masked.txt"):
        f = np.array([float(v) for v in r[0:4]]).reshape(2, 2)
        m = np.array([float(v) for v in r[4:8]]).reshape(2, 2)
        x, y = float(r[8]), float(r[9])
        got = oracle.gather(f * m, m, x, y, L=L)
        if r[10] == "none":
            assert got is None, (r, got)
        else:
            assert got is not None and abs(got - float(r[10])) < 1e-14, (r, got)


def pin_bilinear_exact_on_bilinear_functions(L):
    """a + b i + c j + d i j is reproduced exactly at any point inside the grid."""
    rng = np.random.default_rng(1)
    a, b, c, d = rng.normal(size=4)
    ii, jj = np.meshgrid(np.arange(7.0), np.arange(9.0), indexing="ij")
    F = a + b * ii + c * jj + d * ii * jj
    ones = np.ones_like(F)
    for _ in range(200):
        q0, q1 = rng.uniform(0, 6), rng.uniform(0, 8)
        got = oracle.gather(F, ones, q0, q1, L=L)
        want = a + b * q0 + c * q1 + d * q0 * q1
        assert got is not None and abs(got - want) < 1e-12, (q0, q1, got, want)


def pin_scatter_golden(L):
    frames = np.array([[[6.0]]], dtype=np.float32)
    W = np.array([[2.0]], dtype=np.float32)
    M = np.ones((1, 1), np.uint8)
    u = np.array([[[0.25]], [[0.5]]])
    delta = np.zeros((1, 2))
    Iref, w = oracle.make_object_map(frames, W, M, u, delta, (2, 2), L=L)
    for r in _rows("scatter_single.txt"):
        i, j, wv, iv = int(r[0]), int(r[1]), float(r[2]), float(r[3])
        assert abs(w[i, j] - wv) < 1e-14 and abs(Iref[i, j] - iv) < 1e-14, (r, w, Iref)


# ---------------------------------------------------------------------------------------
# make_object_map (section "Make reference image")
# ---------------------------------------------------------------------------------------

def _integer_scan(rng, N=9, ny=12, nx=10, R=(40, 44)):
    """Integer map and translations; every value exactly representable in float32."""
    Iref = rng.integers(32, 97, size=R).astype(np.float64) / 64.0
    W = (2.0 ** rng.integers(0, 4, size=(ny, nx))).astype(np.float32)
    M = (rng.random((ny, nx)) > 0.15).astype(np.uint8)
    uy = 9 + np.arange(ny) * 2          # magnification 2 along rows, 1 along columns
    ux = 7 + np.arange(nx)
    u = np.empty((2, ny, nx))
    u[0] = uy[:, None]
    u[1] = ux[None, :]
    delta = np.stack([rng.integers(0, 6, N), rng.integers(-3, 4, N)], axis=1).astype(np.float64)
    frames = np.empty((N, ny, nx), np.float32)
    for n in range(N):
        frames[n] = W * Iref[(u[0] - delta[n, 0]).astype(int), (u[1] - delta[n, 1]).astype(int)]
    return frames, W, M, u, delta, Iref


def pin_omap_integer_identity(L):
    """Integer u - Delta: every frame lands on grid points with weight 1, so I_ref is
    reproduced exactly wherever it is covered, and w = sum of W^2 over the hits."""
    rng = np.random.default_rng(2)
    frames, W, M, u, delta, Iref_true = _integer_scan(rng)
    Iref, w = oracle.make_object_map(frames, W, M, u, delta, Iref_true.shape, L=L)
    hits = np.zeros(Iref_true.shape)
    for n in range(frames.shape[0]):
        qi = (u[0] - delta[n, 0]).astype(int)
        qj = (u[1] - delta[n, 1]).astype(int)
        np.add.at(hits, (qi[M > 0], qj[M > 0]), (W.astype(np.float64) ** 2)[M > 0])
    cov = hits > 0
    assert cov.sum() > 50
    assert np.array_equal(Iref[cov], Iref_true[cov]), np.abs(Iref - Iref_true)[cov].max()
    assert np.array_equal(w, hits)
    assert np.all(Iref[~cov] == 0.0)


def _fractional_scan(rng, N=7, ny=9, nx=11, R=(48, 52), const=None):
    u = np.empty((2, ny, nx))
    u[0] = 12 + 1.37 * np.arange(ny)[:, None] + 0.3 * rng.random((ny, nx))
    u[1] = 10 + 1.61 * np.arange(nx)[None, :] + 0.3 * rng.random((ny, nx))
    delta = rng.uniform(0, 8, size=(N, 2))
    W = rng.integers(20, 200, size=(ny, nx)).astype(np.float32)   # W * const exact in float32
    M = (rng.random((ny, nx)) > 0.1).astype(np.uint8)
    if const is None:
        frames = rng.uniform(10, 300, size=(N, ny, nx)).astype(np.float32)
    else:
        frames = np.broadcast_to(W * np.float32(const), (N, ny, nx)).astype(np.float32)
    return frames, W, M, u, delta, R


def pin_omap_constant_reference(L):
    """I = W c  =>  sum b W (W c) / sum b W^2 = c on every covered cell, for any
    fractional positions and any whitefield."""
    rng = np.random.default_rng(3)
    frames, W, M, u, delta, R = _fractional_scan(rng, const=0.75)
    Iref, w = oracle.make_object_map(frames, W, M, u, delta, R, L=L)
    cov = w > 0
    assert cov.sum() > 100
    np.testing.assert_allclose(Iref[cov], 0.75, rtol=1e-12)


def pin_omap_moments(L):
    """The bilinear weights sum to 1 and their centroid is the point itself, so with every
    corner inside the grid: sum w = sum M W^2, sum I_ref w = sum M W I, and
    sum_c c w(c) = sum M W^2 (u - Delta) on each axis."""
    rng = np.random.default_rng(4)
    frames, W, M, u, delta, R = _fractional_scan(rng)
    Iref, w = oracle.make_object_map(frames, W, M, u, delta, R, L=L)
    Wd, Md, Fd = W.astype(np.float64), M.astype(np.float64), frames.astype(np.float64)
    N = frames.shape[0]
    np.testing.assert_allclose(w.sum(), N * (Md * Wd ** 2).sum(), rtol=1e-12)
    np.testing.assert_allclose((Iref * w).sum(), (Md * Wd * Fd).sum(), rtol=1e-12)
    ci, cj = np.meshgrid(np.arange(R[0]), np.arange(R[1]), indexing="ij")
    for axis, cc in ((0, ci), (1, cj)):
        want = sum((Md * Wd ** 2 * (u[axis] - delta[n, axis])).sum() for n in range(N))
        np.testing.assert_allclose((cc * w).sum(), want, rtol=1e-12)


# ---------------------------------------------------------------------------------------
# update_pixel_map (section "Update pixel mapping")
# ---------------------------------------------------------------------------------------

def _direct_window(frames, W, Iref, w, delta, u, window, i, j):
    """e over the window by plain indexing (integer translations only): frames whose
    sample c - Delta_n is outside the grid or uncovered are left out of both sums."""
    Sy, Sx = window
    ci = int(np.floor(u[0, i, j] + 0.5))
    cj = int(np.floor(u[1, i, j] + 0.5))
    e = np.empty((2 * Sy + 1, 2 * Sx + 1))
    Wv = float(W[i, j])
    for a in range(-Sy, Sy + 1):
        for b in range(-Sx, Sx + 1):
            err = var = 0.0
            nv = 0
            for n in range(frames.shape[0]):
                qi, qj = ci + a - int(delta[n, 0]), cj + b - int(delta[n, 1])
                if not (0 <= qi < Iref.shape[0] and 0 <= qj < Iref.shape[1]) or w[qi, qj] <= 0:
                    continue
                I = float(frames[n, i, j])
                err += (I - Wv * Iref[qi, qj]) ** 2
                var += (I - Wv) ** 2
                nv += 1
            e[a + Sy, b + Sx] = np.inf if nv == 0 else (err / var if var > 0 else err)
    return e, (ci, cj)


def pin_upm_window_by_indexing(L):
    rng = np.random.default_rng(5)
    frames, W, M, u, delta, Iref = _integer_scan(rng)
    frames = rng.poisson(frames.astype(np.float64) * 50).astype(np.float32)
    W = (W * 50).astype(np.float32)
    u = u + rng.uniform(-0.49, 0.49, size=u.shape)
    w = np.ones_like(Iref)
    w[20:24, 15:30] = 0.0                     # a hole: frames landing there drop out
    window = (2, 3)
    for (i, j) in [(0, 0), (5, 4), (11, 9), (7, 2), (3, 8)]:
        e, c = oracle.pixel_window(frames, W, M, Iref, w, delta, u, window, i * frames.shape[2] + j, L=L)
        want, cw = _direct_window(frames, W, Iref, w, delta, u, window, i, j)
        assert c == cw, (c, cw)
        np.testing.assert_allclose(e, want, rtol=1e-12)


def _bruteforce_window(frames, W, Iref, w, delta, u, window, i, j):
    """e over the window by a literal loop over "Update pixel mapping" with fractional
    translations: R_n(c) is the masked, renormalised bilinear read at c - Delta_n ("Sub-pixel
    interpolation": corners inside the grid with w > 0 and a nonzero weight count, their
    weights renormalised), a frame with no such corner is left out of both sums."""
    Sy, Sx = window
    Ry, Rx = Iref.shape
    ci = int(np.floor(u[0, i, j] + 0.5))
    cj = int(np.floor(u[1, i, j] + 0.5))
    Wv = float(W[i, j])
    e = np.empty((2 * Sy + 1, 2 * Sx + 1))
    for a in range(-Sy, Sy + 1):
        for b in range(-Sx, Sx + 1):
            err = var = 0.0
            nv = 0
            for n in range(frames.shape[0]):
                p0, p1 = ci + a - float(delta[n, 0]), cj + b - float(delta[n, 1])
                f0, f1 = int(np.floor(p0)), int(np.floor(p1))
                t0, t1 = p0 - f0, p1 - f1
                num = den = 0.0
                for (di, dj, wt) in ((0, 0, (1 - t0) * (1 - t1)), (0, 1, (1 - t0) * t1),
                                     (1, 0, t0 * (1 - t1)), (1, 1, t0 * t1)):
                    qi, qj = f0 + di, f1 + dj
                    if wt == 0.0 or not (0 <= qi < Ry and 0 <= qj < Rx) or w[qi, qj] <= 0:
                        continue
                    num += wt * float(Iref[qi, qj])
                    den += wt
                if den <= 0.0:
                    continue
                I = float(frames[n, i, j])
                err += (I - Wv * num / den) ** 2
                var += (I - Wv) ** 2
                nv += 1
            e[a + Sy, b + Sx] = np.inf if nv == 0 else (err / var if var > 0 else err)
    return e, (ci, cj)


def pin_upm_window_bruteforce_fractional(L):
    """The window errors of a few pixels, fractional translations on both axes and an
    uncovered patch (frames partly and wholly invalid), by a literal loop on tiny inputs."""
    rng = np.random.default_rng(11)
    frames, W, M, u, delta, R = _fractional_scan(rng)
    Iref = rng.uniform(0.5, 1.5, size=R)
    w = rng.uniform(0.5, 2.0, size=R)
    w[20:23, 25:40] = 0.0
    w[30, :] = 0.0
    window = (2, 3)
    for (i, j) in [(0, 0), (4, 5), (8, 10), (6, 2), (2, 9), (5, 7)]:
        e, c = oracle.pixel_window(frames, W, M, Iref, w, delta, u, window, i * frames.shape[2] + j, L=L)
        want, cw = _bruteforce_window(frames, W, Iref, w, delta, u, window, i, j)
        assert c == cw, (c, cw)
        assert np.array_equal(np.isinf(e), np.isinf(want))
        fin = np.isfinite(want)
        np.testing.assert_allclose(e[fin], want[fin], rtol=1e-12)


def pin_upm_exact_search(L):
    """Noiseless frames rendered from the grid at integer positions: the error at the
    truth is 0 and the argmin lands on the truth, starting anywhere in the window."""
    rng = np.random.default_rng(6)
    frames, W, M, u_true, delta, Iref = _integer_scan(rng)
    w = np.ones_like(Iref)
    u0 = u_true + rng.integers(-2, 3, size=u_true.shape) + rng.uniform(-0.4, 0.4, size=u_true.shape)
    u, err = oracle.update_pixel_map(frames, W, M, Iref, w, delta, u0, (3, 3), quadratic=False, L=L)
    good = M > 0
    assert np.array_equal(u[:, good], u_true[:, good])
    assert np.all(err[good] == 0.0)
    assert np.array_equal(u[:, ~good], u0[:, ~good])          # M = 0 keeps its u
    assert np.all(np.isnan(err[~good]))


def pin_upm_linear_field_exact(L):
    """Reference linear along the columns: the error is exactly quadratic in the column
    shift (bilinear reads of a linear function are exact, even at fractional
    translations), so the refined column coordinate equals the truth."""
    rng = np.random.default_rng(7)
    N, ny, nx, R = 6, 5, 7, (30, 60)
    alpha, beta = 0.4, 0.013
    Iref = alpha + beta * np.broadcast_to(np.arange(R[1], dtype=np.float64), R)
    u = np.empty((2, ny, nx))
    u[0] = 10 + np.arange(ny)[:, None]
    u[1] = 15 + 1.3 * np.arange(nx)[None, :] + rng.uniform(-0.45, 0.45, (ny, nx))
    delta = np.stack([np.zeros(N), rng.uniform(0, 9, N)], axis=1)
    W = rng.uniform(50, 150, (ny, nx))
    frames = np.stack([W * (alpha + beta * (u[1] - delta[n, 1])) for n in range(N)])
    frames32 = frames.astype(np.float32)
    # float32 frames: compare against the exact shift of the rounded data
    W32 = W.astype(np.float32)
    M = np.ones((ny, nx), np.uint8)
    u0 = u.copy()
    u0[1] += rng.integers(-2, 3, (ny, nx))
    # a one-row window: the error does not depend on the row, so rows are not searched
    got, err = oracle.update_pixel_map(frames32, W32, M, Iref, np.ones(R), delta, u0, (0, 4),
                                       quadratic=True, L=L)
    np.testing.assert_array_equal(got[0], u[0])
    np.testing.assert_allclose(got[1], u[1], atol=2e-6)


def pin_upm_tie_break(L):
    """Reference periodic with period 2 along the columns and constant along the rows:
    every candidate with the right column parity has error 0; the first one in row-major
    window order (smallest row offset, then smallest column offset) must win."""
    N, ny, nx, R = 4, 3, 4, (30, 40)
    Iref = 1.0 + 0.5 * (np.arange(R[1]) % 2)[None, :] * np.ones((R[0], 1))
    u = np.empty((2, ny, nx))
    u[0] = 12 + np.arange(ny)[:, None]
    u[1] = 15 + np.arange(nx)[None, :]
    delta = np.array([[0, 0], [1, 2], [2, 4], [0, 6]], dtype=np.float64)
    W = np.full((ny, nx), 100.0, np.float32)
    frames = np.stack([W * Iref[(u[0] - d[0]).astype(int), (u[1] - d[1]).astype(int)] for d in delta]).astype(np.float32)
    M = np.ones((ny, nx), np.uint8)
    got, err = oracle.update_pixel_map(frames, W, M, Iref, np.ones(R), delta, u, (2, 3), quadratic=False, L=L)
    # column offsets -3..3 with even offset give error 0; first is -2; row offset -2 wins
    np.testing.assert_array_equal(got[0], u[0] - 2)
    np.testing.assert_array_equal(got[1], u[1] - 2)


def pin_upm_degenerate(L):
    """No valid frame for any candidate: e = +inf everywhere and u is kept."""
    N, ny, nx, R = 3, 2, 2, (10, 10)
    frames = np.full((N, ny, nx), 100, np.float32)
    W = np.full((ny, nx), 90, np.float32)
    M = np.ones((ny, nx), np.uint8)
    u = np.full((2, ny, nx), 5.2)
    delta = np.zeros((N, 2))
    got, err = oracle.update_pixel_map(frames, W, M, np.ones(R), np.zeros(R), delta, u, (1, 1), L=L)
    assert np.array_equal(got, u) and np.all(np.isinf(err))


def pin_reference_terms(L):
    """Integer translations: T[c] = sum over frames whose sample c - Delta_n is inside
    and covered of I_ref[c - Delta_n]^2, counted by plain indexing; fractional
    translations of a constant reference give T = n_valid * const^2."""
    rng = np.random.default_rng(9)
    R = (14, 17)
    Iref = rng.uniform(0.5, 1.5, R)
    w = (rng.random(R) > 0.2).astype(np.float64)
    delta = np.array([[0, 0], [2, -1], [-3, 4], [5, 5], [1, 9]], dtype=np.float64)
    T, nv = oracle.reference_terms(Iref, w, delta, L=L)
    for cy in range(R[0]):
        for cx in range(R[1]):
            t, k = 0.0, 0
            for d in delta.astype(int):
                qy, qx = cy - d[0], cx - d[1]
                if 0 <= qy < R[0] and 0 <= qx < R[1] and w[qy, qx] > 0:
                    t += Iref[qy, qx] ** 2
                    k += 1
            assert nv[cy, cx] == k and abs(T[cy, cx] - t) < 1e-12, (cy, cx)
    frac = rng.uniform(-3, 3, (6, 2))
    T, nv = oracle.reference_terms(np.full(R, 0.8), np.ones(R), frac, L=L)
    np.testing.assert_allclose(T, nv * 0.64, rtol=1e-12)
    assert nv.max() == 6 and nv.min() >= 0


# ---------------------------------------------------------------------------------------
# quadratic refinement
# ---------------------------------------------------------------------------------------

def pin_fit_exact_paraboloid(L):
    rng = np.random.default_rng(8)
    a, b = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0], indexing="ij")
    for _ in range(100):
        A = rng.normal(size=(2, 2))
        H = A @ A.T + 0.2 * np.eye(2)                     # positive definite
        v = rng.uniform(-0.5, 0.5, 2)
        f0 = rng.uniform(0, 3)
        d = np.stack([a - v[0], b - v[1]])
        f = f0 + 0.5 * np.einsum("i...,ij,j...->...", d, H, d)
        da, db = oracle.quadratic_fit(f, L=L)
        assert abs(da - v[0]) < 1e-10 and abs(db - v[1]) < 1e-10, (da, db, v)


def pin_fit_fallbacks(L):
    # a missing corner: the separable parabola is fitted per axis through the cross
    f = np.array([[np.inf, 1.0, 2.0], [0.5, 0.1, 0.9], [2.0, 0.6, 2.0]])
    da, db = oracle.quadratic_fit(f, L=L)
    assert abs(da - (1.0 - 0.6) / (2 * (1.0 - 0.2 + 0.6))) < 1e-14
    assert abs(db - (0.5 - 0.9) / (2 * (0.5 - 0.2 + 0.9))) < 1e-14
    # flat along one axis and a saddle overall: no shift on the flat axis
    f = np.array([[1.0, 0.0, 1.0], [1.0, 0.0, 1.0], [1.0, 0.0, 1.0]])
    assert oracle.quadratic_fit(f, L=L) == (0.0, 0.0)
    # an edge argmin (missing neighbours on one axis only)
    f = np.array([[np.inf, np.inf, np.inf], [0.7, 0.2, 0.3], [0.9, 0.5, 0.8]])
    da, db = oracle.quadratic_fit(f, L=L)
    assert da == 0.0 and abs(db - (0.7 - 0.3) / (2 * (0.7 - 0.4 + 0.3))) < 1e-14


# ---------------------------------------------------------------------------------------
# truth recovery on noiseless data with the true reference
# ---------------------------------------------------------------------------------------

def pin_truth_recovery(L):
    """400 frames of noiseless data rendered from the continuous field (not from its
    grid), the grid as I_ref: one update recovers the fractional truth to 0.01 px RMS
    with no bias beyond 0.002 px."""
    s = gen.tiny2d(n_side=20, det=32, step=2, ref=120, sigma=2.0, mag=1.5, offset=50.0,
                   aberr=3.0, noise=False, seed=gen.BASE_SEED + 100)
    u, err = oracle.update_pixel_map(s.frames, s.W, s.M, s.Iref_true, np.ones(s.ref_shape), s.delta,
                                     s.u_true, s.window, L=L)
    d = (u - s.u_true)[:, 2:-2, 2:-2]
    rms = float(np.sqrt((d ** 2).mean()))
    assert rms < 0.01, rms
    assert abs(float(d.mean())) < 0.002, d.mean()
    assert float(np.abs(d).max()) < 0.05, np.abs(d).max()


# ---------------------------------------------------------------------------------------
# figures of merit (section "Calculate figures of merit")
# ---------------------------------------------------------------------------------------

def pin_error_exact_zero(L):
    """Integer map and translations with frames W * I_ref exactly: every error term is 0,
    so the pixel, frame, total and reference-plane errors are exactly 0 (M = 0: NaN)."""
    rng = np.random.default_rng(31)
    frames, W, M, u, delta, Iref = _integer_scan(rng)
    pe, fe, tot, re = oracle.calc_error(frames, W, M, Iref, np.ones(Iref.shape), u, delta, L=L)
    assert np.all(pe[M > 0] == 0.0) and np.all(np.isnan(pe[M == 0]))
    assert np.all(fe == 0.0) and tot == 0.0 and np.all(re == 0.0)


def pin_error_matches_search_error(L):
    """At an integer map the pixel error is the update step's normalised error of the
    candidate at the window centre (pinned separately), and the sums agree: sum of pixel
    errors = sum of frame errors = total."""
    rng = np.random.default_rng(32)
    frames, W, M, u, delta, Iref = _integer_scan(rng)
    frames = frames * np.float32(1.0) + rng.uniform(-0.2, 0.2, frames.shape).astype(np.float32)
    w = np.ones(Iref.shape)
    w[18:22, 20:25] = 0.0                                    # a hole: some frames invalid
    pe, fe, tot, re = oracle.calc_error(frames, W, M, Iref, w, u, delta, L=L)
    ny, nx = M.shape
    checked = 0
    for p in range(ny * nx):
        if not M.flat[p]:
            continue
        e, _ = oracle.pixel_window(frames, W, M, Iref, w, delta, u, (0, 0), p, L=L)
        if np.isfinite(e[0, 0]):
            np.testing.assert_allclose(pe.flat[p], e[0, 0], rtol=1e-12, atol=1e-15)
            checked += 1
    assert checked > 50
    np.testing.assert_allclose(np.nansum(pe), tot, rtol=1e-12)
    np.testing.assert_allclose(fe.sum(), tot, rtol=1e-12)


def pin_error_reference_plane_weights(L):
    """Fully covered reference, all reads inside the grid: every frame of every pixel is
    valid, so the weights landing on each reference pixel are make_object_map's w for unit
    frames and whitefield (pinned separately); the reference-plane error weighted by them
    sums to the total error."""
    rng = np.random.default_rng(33)
    frames, W, M, u, delta, R = _fractional_scan(rng)
    Iref = rng.uniform(0.5, 1.5, R)
    w = np.ones(R)
    pe, fe, tot, re = oracle.calc_error(frames, W, M, Iref, w, u, delta, L=L)
    ones = np.ones_like(frames)
    _, den = oracle.make_object_map(ones, np.ones_like(W), M, u, delta, R, L=L)
    np.testing.assert_allclose((re * den).sum(), tot, rtol=1e-11)
    assert np.all(re[den == 0] == 0.0)


# ---------------------------------------------------------------------------------------
# update_translations (section "Update translations")
# ---------------------------------------------------------------------------------------

def pin_translations_exact_integer(L):
    """Frames W * I_ref(u - Delta) exactly, integer everything, I_ref random: the error is 0
    at the true translation and positive elsewhere, so starting from integer offsets inside
    the window every translation is recovered exactly (no fit)."""
    rng = np.random.default_rng(34)
    frames, W, M, u, delta, Iref = _integer_scan(rng, N=6)
    start = delta + rng.integers(-2, 3, size=delta.shape)
    got, err = oracle.update_translations(frames, W, M, Iref, np.ones(Iref.shape), u, start, (3, 3),
                                          quadratic=False, L=L)
    np.testing.assert_array_equal(got, delta)
    assert np.all(err == 0.0)


def pin_translations_window_by_indexing(L):
    """A frame's error window for integer shifts, computed by plain array indexing: the mean
    over good pixels of (I - W I_ref[u - Delta - t])^2 / var, var over the frames at the
    current translations."""
    rng = np.random.default_rng(35)
    frames, W, M, u, delta, Iref = _integer_scan(rng, N=5)
    frames = frames + rng.uniform(-0.3, 0.3, frames.shape).astype(np.float32)
    Ry, Rx = Iref.shape
    ui, uj = u[0].astype(int), u[1].astype(int)
    F, Wd = frames.astype(np.float64), W.astype(np.float64)
    var = np.zeros(M.shape)
    for n in range(frames.shape[0]):
        var += (F[n] - Wd) ** 2                           # every read is on the grid here
    T = 2
    for n in (0, 3):
        e = oracle.frame_window(frames, W, M, Iref, np.ones(Iref.shape), u, delta, (T, T), n, L=L)
        for a in range(-T, T + 1):
            for b in range(-T, T + 1):
                qi, qj = ui - int(delta[n, 0]) - a, uj - int(delta[n, 1]) - b
                ok = (M > 0) & (qi >= 0) & (qi < Ry) & (qj >= 0) & (qj < Rx) & (var > 0)
                R = Iref[np.clip(qi, 0, Ry - 1), np.clip(qj, 0, Rx - 1)]
                want = (((F[n] - Wd * R) ** 2) / np.where(var > 0, var, 1.0))[ok].mean()
                np.testing.assert_allclose(e[a + T, b + T], want, rtol=1e-12)


def pin_translations_linear_field_exact(L):
    """Reference linear along the columns and translations along the columns only: a
    frame's error is exactly quadratic in the column shift, so the refined translation
    equals the truth from a fractional start."""
    rng = np.random.default_rng(36)
    N, ny, nx, R = 5, 6, 9, (30, 70)
    alpha, beta = 0.4, 0.011
    Iref = alpha + beta * np.broadcast_to(np.arange(R[1], dtype=np.float64), R)
    u = np.empty((2, ny, nx))
    u[0] = 10 + np.arange(ny)[:, None]
    u[1] = 20 + 1.3 * np.arange(nx)[None, :] + rng.uniform(-0.45, 0.45, (ny, nx))
    delta = np.stack([np.zeros(N), rng.uniform(0, 9, N)], axis=1)
    W = rng.uniform(50, 150, (ny, nx))
    frames = np.stack([W * (alpha + beta * (u[1] - delta[n, 1])) for n in range(N)]).astype(np.float64)
    M = np.ones((ny, nx), np.uint8)
    start = delta.copy()
    start[:, 1] += rng.uniform(-1.4, 1.4, N)
    # float32 frames: the truth of the rounded data differs from delta by ~1e-6
    got, err = oracle.update_translations(frames.astype(np.float32), W.astype(np.float32), M, Iref, np.ones(R), u,
                                          start, (0, 3), quadratic=True, L=L)
    np.testing.assert_array_equal(got[:, 0], delta[:, 0])
    np.testing.assert_allclose(got[:, 1], delta[:, 1], atol=5e-5)


# ---------------------------------------------------------------------------------------
# regularisation of the pixel map (the "sigma" option of the update)
# ---------------------------------------------------------------------------------------

def pin_filter_scipy(L):
    """The normalised Gaussian filter equals scipy's separable gaussian_filter of M u and of M
    (zero outside the detector, the same 4-sigma truncation), divided."""
    import scipy.ndimage as ndi
    rng = np.random.default_rng(41)
    ny, nx, sigma = 23, 31, 1.7
    M = (rng.random((ny, nx)) > 0.2).astype(np.uint8)
    u = np.stack([100 + rng.normal(0, 3, (ny, nx)), 50 + rng.normal(0, 3, (ny, nx))])
    got = oracle.filter_map(M, u, sigma, L=L)
    m = M.astype(np.float64)
    kw = dict(sigma=sigma, mode="constant", cval=0.0, truncate=4.0)
    den = ndi.gaussian_filter(m, **kw)
    for c in range(2):
        want = ndi.gaussian_filter(m * u[c], **kw) / den
        np.testing.assert_allclose(got[c][M > 0], want[M > 0], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(got[c][M == 0], u[c][M == 0])


def pin_filter_preserves_linear_and_constant(L):
    """A constant map is unchanged; a linear map is unchanged at pixels whose whole kernel
    support is inside the detector and unmasked (a symmetric kernel averages a linear
    function to its centre); sigma = 0 is the identity."""
    ny, nx, sigma = 30, 40, 2.0
    M = np.ones((ny, nx), np.uint8)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    u = np.stack([7.0 + 1.3 * y + 0.2 * x, -3.0 + 0.7 * x - 0.1 * y])
    got = oracle.filter_map(M, u, sigma, L=L)
    r = int(np.floor(4 * sigma + 0.5))
    inner = (slice(r, ny - r), slice(r, nx - r))
    np.testing.assert_allclose(got[0][inner], u[0][inner], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got[1][inner], u[1][inner], rtol=0, atol=1e-11)
    c = np.full((2, ny, nx), 123.456)
    np.testing.assert_allclose(oracle.filter_map(M, c, sigma, L=L), c, rtol=1e-14)
    np.testing.assert_array_equal(oracle.filter_map(M, u, 0.0, L=L), u)


# ---------------------------------------------------------------------------------------
# fractional candidates (the non-integer option of section "Update pixel mapping")
# ---------------------------------------------------------------------------------------

def _bilinear_np(Iref, q0, q1):
    """Plain bilinear interpolation of a fully covered grid (independent of the oracle)."""
    i0, j0 = np.floor(q0).astype(int), np.floor(q1).astype(int)
    fy, fx = q0 - i0, q1 - j0
    return ((1 - fy) * (1 - fx) * Iref[i0, j0] + (1 - fy) * fx * Iref[i0, j0 + 1] +
            fy * (1 - fx) * Iref[i0 + 1, j0] + fy * fx * Iref[i0 + 1, j0 + 1])


def pin_frac_exact_on_bilinear_data(L):
    """Frames rendered by bilinear reads of the grid reference at maps on a quarter-pixel
    grid: the error vanishes at the true map, so the quarter-pixel search recovers it
    exactly (and a unit step, sub = 1, leaves the integer search's answer)."""
    import scipy.ndimage as ndi
    rng = np.random.default_rng(51)
    N, ny, nx, R = 16, 7, 8, (40, 44)
    # a speckle-like reference (correlated over ~2 pixels), so that the integer search's
    # minimum lies next to the true map
    Iref = ndi.gaussian_filter(rng.random(R), 1.5, mode="wrap")
    Iref = 0.5 + (Iref - Iref.min()) / (Iref.max() - Iref.min())
    u = np.empty((2, ny, nx))
    u[0] = 12 + np.arange(ny)[:, None] * 1.5 + rng.integers(0, 4, (ny, nx)) / 4.0
    u[1] = 10 + np.arange(nx)[None, :] * 1.25 + rng.integers(0, 4, (ny, nx)) / 4.0
    delta = np.stack([rng.integers(0, 6, N), rng.integers(-3, 4, N)], axis=1).astype(np.float64)
    W = rng.uniform(200, 400, (ny, nx))
    frames = np.stack([W * _bilinear_np(Iref, u[0] - delta[n, 0], u[1] - delta[n, 1]) for n in range(N)])
    M = np.ones((ny, nx), np.uint8)
    start = np.round(u)
    got, err = oracle.update_pixel_map_frac(frames.astype(np.float32), W.astype(np.float32), M, Iref, np.ones(R),
                                            delta, start, (2, 2), 4, L=L)
    np.testing.assert_array_equal(got, u)
    ui, ei = oracle.update_pixel_map(frames.astype(np.float32), W.astype(np.float32), M, Iref, np.ones(R), delta,
                                     start, (2, 2), quadratic=False, L=L)
    g1, e1 = oracle.update_pixel_map_frac(frames.astype(np.float32), W.astype(np.float32), M, Iref, np.ones(R),
                                          delta, start, (2, 2), 1, L=L)
    # sub = 1: the integer minimum's 3x3, whose first minimum is that minimum unless a
    # neighbour ties it exactly
    assert np.mean(np.all(g1 == ui, axis=0)) > 0.95
    assert np.all(e1 <= ei)


# ---------------------------------------------------------------------------------------
# defocus registration (fit_defocus_registration, section "Initialisation")
# ---------------------------------------------------------------------------------------

def pin_defocus_contrast_definition(L):
    """Unit scales give make_object_map's reference image (pinned separately), whose contrast
    is numpy's std / mean over the covered pixels; constant frames have contrast 0 at every
    scale."""
    rng = np.random.default_rng(61)
    frames, W, M, u, delta, R = _fractional_scan(rng)
    got = oracle.defocus_sweep(frames, W, M, u, delta, R, [1.0], [1.0], L=L)
    Iref, w = oracle.make_object_map(frames, W, M, u, delta, R, L=L)
    cov = w > 0
    np.testing.assert_allclose(got[0, 0], Iref[cov].std() / Iref[cov].mean(), rtol=1e-12)
    fr_c, W_c, M_c, u_c, d_c, R_c = _fractional_scan(rng, const=0.75)
    sweep = oracle.defocus_sweep(fr_c, W_c, M_c, u_c, d_c, R_c, [0.97, 1.0, 1.03], [0.98, 1.02], L=L)
    assert np.all(np.abs(sweep) < 1e-12), sweep


def pin_defocus_recovers_magnification(L):
    """Noiseless frames rendered from the continuous field at the true magnification, a base
    map with the wrong one: the sweep's contrast is highest at the scale that restores the
    true magnification on each axis."""
    # translations spanning 36 pixels, so that a 2 % scale error misregisters the frames by
    # a good fraction of the speckle size
    s = gen.tiny2d(n_side=4, det=48, step=12, ref=170, sigma=1.5, mag=1.4, offset=50.0, aberr=0.0, window=3,
                   seed=gen.BASE_SEED + 63, noise=False)
    # the base map: slopes 4 % too small on rows and 4 % too large on columns
    ny, nx = s.M.shape
    pc = (ny // 2, nx // 2)
    u = s.u_true.copy()
    u[0] = u[0][pc] + (1 / 1.04) * (u[0] - u[0][pc])
    u[1] = u[1][pc] + (1 / 0.96) * (u[1] - u[1][pc])
    sy = np.array([0.98, 1.00, 1.02, 1.04, 1.06, 1.08])
    sx = np.array([0.92, 0.94, 0.96, 0.98, 1.00, 1.02])
    c = oracle.defocus_sweep(s.frames, s.W, s.M, u, s.delta, s.ref_shape, sy, sx, L=L)
    ky, kx = np.unravel_index(np.argmax(c), c.shape)
    assert (sy[ky], sx[kx]) == (1.04, 0.96), (sy[ky], sx[kx], c)


# ---- the "integrate" option (R17) ------------------------------------------------------
def _integ_masks():
    """A full detector, one with isolated bad pixels and a notch, one with a bad border row."""
    full = np.ones((18, 23), np.uint8)
    holes = full.copy()
    holes[4, 6] = holes[9, 15] = holes[13, 3] = 0
    holes[0:3, 19:] = 0
    edge = full.copy()
    edge[:, 0] = 0
    edge[17, :] = 0
    return [full, holes, edge]


def pin_integrate_quadratic_potential_unchanged(L):
    """The gradient of a quadratic potential is a fixed point: every stencil the reading uses
    where at least two neighbours are good is exact for quadratics."""
    i, j = np.mgrid[0:18, 0:23].astype(np.float64)
    # Psi = 104 i + 37 j + 0.51 i^2 + 0.03 i j + 0.49 j^2 (a magnification ~1 and a rotation-free shear)
    u = np.stack([104.0 + 1.02 * i + 0.03 * j, 37.0 + 0.03 * i + 0.98 * j])
    for M in _integ_masks():
        out, it, res = oracle.integrate_map(M, u, tol=1e-13, L=L)
        assert res < 1e-12
        assert np.abs(out - u)[:, M > 0].max() < 1e-7, np.abs(out - u)[:, M > 0].max()


def pin_integrate_is_an_orthogonal_projection(L):
    """Least squares onto gradient fields is an orthogonal projection P: P(P u) = P u,
    <u - P u, P w> = 0 and <P u, w> = <u, P w> for any maps u, w (the entries without an
    equation, where P leaves the map, cancel on both sides), and P is linear."""
    rng = np.random.default_rng(12726 + 501)
    for M in _integ_masks():
        u = rng.normal(size=(2,) + M.shape)
        w = rng.normal(size=(2,) + M.shape)
        Pu, _, r1 = oracle.integrate_map(M, u, tol=1e-13, L=L)
        Pw, _, r2 = oracle.integrate_map(M, w, tol=1e-13, L=L)
        PPu, _, _ = oracle.integrate_map(M, Pu, tol=1e-13, L=L)
        assert r1 < 1e-12 and r2 < 1e-12
        assert np.abs(PPu - Pu).max() < 1e-8
        assert abs(np.sum((u - Pu) * Pw)) < 1e-8 * np.sum(u * u) ** 0.5 * np.sum(w * w) ** 0.5
        assert abs(np.sum(Pu * w) - np.sum(u * Pw)) < 1e-8 * np.sum(u * u) ** 0.5 * np.sum(w * w) ** 0.5
        Pl, _, _ = oracle.integrate_map(M, 2.0 * u - 3.0 * w, tol=1e-13, L=L)
        assert np.abs(Pl - (2.0 * Pu - 3.0 * Pw)).max() < 1e-8


def pin_integrate_output_is_curl_free(L):
    """On a full detector the output's curl by central differences vanishes at every pixel
    two or more from the border (there the output is a central-difference gradient, and
    central differences along the two axes commute)."""
    rng = np.random.default_rng(12726 + 502)
    M = np.ones((20, 26), np.uint8)
    u = rng.normal(size=(2, 20, 26)) * 3.0
    out, _, res = oracle.integrate_map(M, u, tol=1e-13, L=L)
    assert res < 1e-12
    d_u1_di = 0.5 * (out[1][2:, 1:-1] - out[1][:-2, 1:-1])
    d_u0_dj = 0.5 * (out[0][1:-1, 2:] - out[0][1:-1, :-2])
    curl = (d_u1_di - d_u0_dj)[1:-1, 1:-1]
    assert np.abs(curl).max() < 1e-8
    # and the input had a curl of order one
    raw = 0.5 * (u[1][2:, 1:-1] - u[1][:-2, 1:-1]) - 0.5 * (u[0][1:-1, 2:] - u[0][1:-1, :-2])
    assert np.abs(raw).max() > 1.0


def pin_integrate_removes_a_pure_curl(L):
    """A divergence-free field with no flux through the border (the rotated gradient of a
    stream function that vanishes there) is orthogonal to every gradient field: the
    projection removes it, up to the discretisation of the stencils."""
    ny, nx = 40, 48
    i, j = np.mgrid[0:ny, 0:nx].astype(np.float64)
    # stream function s = sin(pi i / (ny - 1))^2 sin(pi j / (nx - 1))^2; u = (ds/dj, -ds/di)
    a, b = np.pi / (ny - 1), np.pi / (nx - 1)
    ds_di = 2 * a * np.sin(a * i) * np.cos(a * i) * np.sin(b * j) ** 2
    ds_dj = 2 * b * np.sin(b * j) * np.cos(b * j) * np.sin(a * i) ** 2
    u = np.stack([ds_dj, -ds_di]) * 50.0
    M = np.ones((ny, nx), np.uint8)
    out, _, res = oracle.integrate_map(M, u, tol=1e-13, L=L)
    assert res < 1e-12
    assert np.sqrt(np.mean(out ** 2)) < 0.03 * np.sqrt(np.mean(u ** 2)), np.sqrt(np.mean(out ** 2))


def pin_integrate_bruteforce(L):
    """A tiny detector with holes: the output equals the least-squares solution computed by
    numpy.linalg.lstsq on the equations written out as a dense matrix, one row per good pixel
    and axis with a good neighbour (central difference, else the second-order one-sided
    difference forward then backward, else the first-order one forward then backward)."""
    rng = np.random.default_rng(12726 + 503)
    M = np.ones((6, 7), np.uint8)
    M[2, 3] = 0
    M[0, 0] = 0
    M[5, 5:] = 0
    ny, nx = M.shape
    u = rng.normal(size=(2, ny, nx)) * 2.0 + 5.0
    good = lambda y, x: 0 <= y < ny and 0 <= x < nx and M[y, x] > 0
    rows, rhs, where = [], [], []
    for a in (0, 1):
        for y in range(ny):
            for x in range(nx):
                if not M[y, x]:
                    continue
                e = (1, 0) if a == 0 else (0, 1)
                at = lambda k: (y + k * e[0], x + k * e[1])
                if good(*at(1)) and good(*at(-1)):
                    taps = [(at(1), 0.5), (at(-1), -0.5)]
                elif good(*at(1)) and good(*at(2)):
                    taps = [(at(0), -1.5), (at(1), 2.0), (at(2), -0.5)]
                elif good(*at(-1)) and good(*at(-2)):
                    taps = [(at(0), 1.5), (at(-1), -2.0), (at(-2), 0.5)]
                elif good(*at(1)):
                    taps = [(at(1), 1.0), (at(0), -1.0)]
                elif good(*at(-1)):
                    taps = [(at(0), 1.0), (at(-1), -1.0)]
                else:
                    continue
                row = np.zeros(ny * nx)
                for (yy, xx), c in taps:
                    row[yy * nx + xx] += c
                rows.append(row)
                rhs.append(u[a, y, x])
                where.append((a, y, x))
    G = np.array(rows)
    psi = np.linalg.lstsq(G, np.array(rhs), rcond=None)[0]
    want = u.copy()
    for k, (a, y, x) in enumerate(where):
        want[a, y, x] = G[k] @ psi
    out, _, res = oracle.integrate_map(M, u, tol=1e-14, L=L)
    assert np.abs(out - want).max() < 1e-8, np.abs(out - want).max()


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
