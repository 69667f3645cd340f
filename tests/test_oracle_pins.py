"""The oracle against its pins (no GPU)."""
import numpy as np
import pytest

import oracle
import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.lib())


def test_iterate_is_the_two_steps_composed():
    import gen
    s = gen.tiny2d(n_side=3, det=24, ref=90, offset=20.0, window=3, noise=True, seed=gen.BASE_SEED + 7)
    u1, I1, w1, e1 = oracle.iterate(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window, 2)
    u = s.u_init.copy()
    for _ in range(2):
        Iref, w = oracle.make_object_map(s.frames, s.W, s.M, u, s.delta, s.ref_shape)
        u, e = oracle.update_pixel_map(s.frames, s.W, s.M, Iref, w, s.delta, u, s.window)
    assert np.array_equal(u, u1) and np.array_equal(Iref, I1) and np.array_equal(w, w1)
    assert np.array_equal(e, e1, equal_nan=True)


def test_rows_and_pixel_list_agree_with_full_update():
    import gen
    s = gen.tiny2d(n_side=3, det=24, ref=90, offset=20.0, window=3, seed=gen.BASE_SEED + 8)
    Iref, w = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    u_full, e_full = oracle.update_pixel_map(s.frames, s.W, s.M, Iref, w, s.delta, s.u_init, s.window)
    u_rows, e_rows = oracle.update_pixel_map(s.frames, s.W, s.M, Iref, w, s.delta, s.u_init, s.window,
                                             rows=(5, 9), threads=1)
    assert np.array_equal(u_rows[:, 5:9], u_full[:, 5:9])
    assert np.array_equal(u_rows[:, :5], s.u_init[:, :5])
    pix = np.array([0, 17, 24 * 12 + 3, 24 * 24 - 1])
    up, ep = oracle.update_pixels(s.frames, s.W, s.M, Iref, w, s.delta, s.u_init, s.window, pix)
    assert np.array_equal(up.T, u_full.reshape(2, -1)[:, pix])
    assert np.array_equal(ep, e_full.ravel()[pix], equal_nan=True)


def test_iteration_reduces_the_error_and_recovers_the_map():
    """Main loop on the small 2-D workload: the total error falls from the initial map to
    the last iteration and the map moves toward the truth (gauge removed). This is a
    reported behaviour, checked loosely: the paper says convergence is not guaranteed."""
    import gen
    s = gen.config_small()
    u = s.u_init.copy()
    totals = []
    for _ in range(s.n_iter):
        Iref, w = oracle.make_object_map(s.frames, s.W, s.M, u, s.delta, s.ref_shape)
        u, e = oracle.update_pixel_map(s.frames, s.W, s.M, Iref, w, s.delta, u, s.window)
        totals.append(float(np.nansum(e[np.isfinite(e)])))
    assert totals[-1] < totals[0]
    d0 = s.u_init - s.u_true
    d = u - s.u_true
    d0 = d0 - d0.mean(axis=(1, 2), keepdims=True)
    d = d - d.mean(axis=(1, 2), keepdims=True)
    assert np.sqrt((d ** 2).mean()) < np.sqrt((d0 ** 2).mean())
