"""The seeded input generator: deterministic, the conventions the C ABI expects, and the
forward model of the "Initialisation" section (frames = W x the reference at u - Delta)."""
import numpy as np

import gen


def test_seeded_and_deterministic():
    a = gen.tiny2d(n_side=2, det=24, ref=80, offset=20.0, window=3, seed=gen.BASE_SEED + 90)
    b = gen.tiny2d(n_side=2, det=24, ref=80, offset=20.0, window=3, seed=gen.BASE_SEED + 90)
    c = gen.tiny2d(n_side=2, det=24, ref=80, offset=20.0, window=3, seed=gen.BASE_SEED + 91)
    assert np.array_equal(a.frames, b.frames) and np.array_equal(a.Iref_true, b.Iref_true)
    assert not np.array_equal(a.frames, c.frames)


def test_conventions():
    s = gen.tiny2d(n_side=2, det=24, ref=80, offset=20.0, window=3, seed=gen.BASE_SEED + 92)
    n, ny, nx = s.frames.shape
    assert s.frames.dtype == np.float32 and s.W.dtype == np.float32 and s.M.dtype == np.uint8
    assert s.u_true.shape == (2, ny, nx) and s.u_true.dtype == np.float64
    assert s.delta.shape == (n, 2) and s.delta.dtype == np.float64
    assert s.Iref_true.shape == s.ref_shape
    # the grid samples of the field span exactly [0.5, 1.5]
    assert abs(s.Iref_true.min() - 0.5) < 1e-12 and abs(s.Iref_true.max() - 1.5) < 1e-12
    # mask: W at least 5 % of its peak
    assert np.array_equal(s.M, (s.W.astype(np.float64) >= 0.05 * s.W.max()).astype(np.uint8))


def test_noiseless_frames_follow_the_forward_model():
    # magnification 1 and integer maps and translations: every frame sample is a grid
    # sample of the field, so frames = W * Iref_true[u - Delta] exactly (to float32)
    ny = nx = 20
    uy = 30.0 + np.arange(ny)
    ux = 25.0 + np.arange(nx)
    delta = gen.grid_delta(3, 4)
    W = np.full((ny, nx), 500.0)
    s = gen.make_scan("t", ny=ny, nx=nx, ref_shape=(80, 80), sigma=2.0, delta=delta, uy=uy, ux=ux,
                      uy0=uy, ux0=ux, W=W, window=(2, 2), n_iter=1, seed=gen.BASE_SEED + 93, noise=False)
    for n in range(delta.shape[0]):
        iy = (uy - delta[n, 0]).astype(int)
        ix = (ux - delta[n, 1]).astype(int)
        want = (500.0 * s.Iref_true[np.ix_(iy, ix)]).astype(np.float32)
        np.testing.assert_allclose(s.frames[n], want, rtol=1e-6)


def test_point_evaluation_equals_the_separable_one():
    """The field at arbitrary points (every tap summed per point) equals the separable band
    sums on a grid of points, to rounding."""
    f = gen.Field((60, 70), 1.5, np.random.default_rng(gen.BASE_SEED + 94))
    py, px = np.linspace(8, 50, 23), np.linspace(9, 61, 29)
    PY, PX = np.meshgrid(py, px, indexing="ij")
    np.testing.assert_allclose(f.points(PY, PX).reshape(PY.shape), f.separable(py, px), rtol=0, atol=1e-12)


def test_nonseparable_map_and_isolated_bad_pixels():
    s = gen.nonsep2d(n_side=2, det=40, ref=110, seed=gen.BASE_SEED + 95, bad_frac=0.02)
    t = gen.nonsep2d(n_side=2, det=40, ref=110, seed=gen.BASE_SEED + 95, bad_frac=0.02)
    assert np.array_equal(s.frames, t.frames) and np.array_equal(s.M, t.M)
    # the map couples the axes: u_y changes along a row, u_x down a column
    assert np.ptp(s.u_true[0][20]) > 0.5 and np.ptp(s.u_true[1][:, 20]) > 0.5
    # a nonzero curl: d u_x / d y - d u_y / d x = 2 theta plus the shear terms, whose means
    # over whole periods vanish
    curl = np.gradient(s.u_true[1], axis=0) - np.gradient(s.u_true[0], axis=1)
    assert abs(curl.mean() - 2 * 0.03) < 0.01 and np.abs(curl).max() > 0.1
    # bad pixels: about 2 % of the good region, each with 8 good neighbours
    full = (s.W.astype(np.float64) >= 0.05 * s.W.max())
    bad = full & (s.M == 0)
    assert abs(bad.sum() - round(0.02 * full.sum())) <= 1
    for i, j in zip(*np.nonzero(bad)):
        nb = s.M[i - 1:i + 2, j - 1:j + 2].copy()
        nb[1, 1] = 1
        assert nb.all()
    # noiseless frames are W times the field at u_true - Delta
    z = gen.nonsep2d(n_side=2, det=24, ref=90, seed=gen.BASE_SEED + 96, noise=False, bad_frac=0.0)
    f = gen.Field(z.ref_shape, z.sigma, np.random.default_rng(gen.BASE_SEED + 96))
    want = z.W.astype(np.float64) * f.points(z.u_true[0] - z.delta[1, 0], z.u_true[1] - z.delta[1, 1]).reshape(24, 24)
    np.testing.assert_allclose(z.frames[1], want.astype(np.float32), rtol=1e-6)
