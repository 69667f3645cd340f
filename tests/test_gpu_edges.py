"""Edge and degenerate cases of the CUDA path, each against the oracle or a fixed rule."""
import numpy as np
import pytest

import gen
import oracle
import parity
from gpu_util import dev, dims_of, gpu_make_object_map, gpu_update

pytestmark = pytest.mark.gpu


def _check_all(s, Iref64, w64, window, quadratic=True):
    I32, w32 = Iref64.astype(np.float32), w64.astype(np.float32)
    inp = dict(frames=s.frames, W=s.W, M=s.M, Iref=I32.astype(np.float64), w=w32.astype(np.float64),
               delta=s.delta, u=s.u_init, window=window)
    ug_i, eg_i = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, window, quadratic=False)
    ug_q, eg_q = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, window, quadratic=quadratic)
    pix = np.flatnonzero(s.M.ravel())
    return parity.check_update(inp, pix, ug_i.reshape(2, -1)[:, pix], eg_i.ravel()[pix],
                               ug_q.reshape(2, -1)[:, pix], eg_q.ravel()[pix])


def test_single_frame_and_single_candidate():
    s = gen.tiny2d(n_side=1, det=20, ref=70, offset=10.0, window=0, seed=gen.BASE_SEED + 31)
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    Ig, wg = gpu_make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    parity.check_omap(Ig, wg, Io, wo)
    _check_all(s, Io, wo, (0, 0))
    _check_all(s, Io, wo, (0, 3))
    _check_all(s, Io, wo, (2, 0))


def test_one_pixel_detector():
    s = gen.tiny2d(n_side=3, det=1, ref=40, offset=15.0, window=2, seed=gen.BASE_SEED + 32, w_sigma=5.0)
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    Ig, wg = gpu_make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    parity.check_omap(Ig, wg, Io, wo)
    _check_all(s, Io, wo, s.window)


def test_everything_masked_is_a_no_op():
    s = gen.tiny2d(n_side=2, det=24, ref=60, offset=10.0, window=2, seed=gen.BASE_SEED + 33)
    s.M[:] = 0
    Ig, wg = gpu_make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    assert np.all(Ig == 0) and np.all(wg == 0)
    ug, eg = gpu_update(s.frames, s.W, s.M, Ig, wg, s.delta, s.u_init, s.window)
    assert np.array_equal(ug, s.u_init) and np.all(np.isnan(eg))


def test_nothing_covered_keeps_u_and_reports_inf():
    s = gen.tiny2d(n_side=2, det=24, ref=60, offset=10.0, window=2, seed=gen.BASE_SEED + 34)
    I0 = np.zeros(s.ref_shape, np.float32)
    ug, eg = gpu_update(s.frames, s.W, s.M, I0, I0, s.delta, s.u_init, s.window)
    good = s.M > 0
    assert np.array_equal(ug, s.u_init) and np.all(np.isinf(eg[good]))


def test_map_outside_the_reference():
    """Pixels whose whole window falls off the reference keep their map (every candidate
    has no valid frame); their neighbours near the border lose frames individually."""
    s = gen.tiny2d(n_side=3, det=32, ref=100, offset=20.0, window=3, seed=gen.BASE_SEED + 35)
    s.u_init -= 30.0          # a poor initial map: many pixels now point off the reference
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    Ig, wg = gpu_make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    parity.check_omap(Ig, wg, Io, wo)
    rep = _check_all(s, Io, wo, s.window)
    print(rep)


def test_more_frames_than_shared_memory_holds():
    """1500 frames: too many to stage on chip, so every pixel takes the exact path."""
    import paper_2003_12726_gb300 as px
    n_side = 39   # 1521 frames
    s = gen.tiny2d(n_side=n_side, det=8, step=1, ref=90, offset=45.0, window=2,
                   seed=gen.BASE_SEED + 36, w_sigma=8.0)
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    _check_all(s, Io, wo, s.window)


def test_nonfinite_map_sets_the_status_word():
    import paper_2003_12726_gb300 as px
    import torch
    s = gen.tiny2d(n_side=2, det=16, ref=50, offset=10.0, window=2, seed=gen.BASE_SEED + 37)
    u = s.u_init.copy()
    u[0, 3, 4] = np.nan
    u[1, 5, 6] = 1e12
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    d = dims_of(s.frames, s.ref_shape)
    o = px.Options(2, 2, True)
    ws = px.workspace(d, o)
    ud = dev(u, torch.float64)
    px.update_pixel_map(d, o, dev(s.frames, torch.float32), dev(s.W, torch.float32), dev(s.M, torch.uint8),
                        dev(Io, torch.float32), dev(wo, torch.float32), dev(s.delta, torch.float64), ud, None, ws)
    code, bits = px.get_status(ws)
    assert code == -3 and bits & 0x1 and bits & 0x2
    out = ud.cpu().numpy()
    assert np.isnan(out[0, 3, 4]) and out[1, 5, 6] == 1e12       # left untouched
    assert px.get_status(ws) == (0, 0)                             # cleared by the read


def test_host_side_argument_errors():
    import paper_2003_12726_gb300 as px
    import torch
    s = gen.tiny2d(n_side=2, det=16, ref=50, offset=10.0, window=2, seed=gen.BASE_SEED + 38)
    d = dims_of(s.frames, s.ref_shape)
    o = px.Options(2, 2, True)
    small = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    args = [dev(s.frames, torch.float32), dev(s.W, torch.float32), dev(s.M, torch.uint8),
            torch.zeros(s.ref_shape, device="cuda"), torch.ones(s.ref_shape, device="cuda"),
            dev(s.delta, torch.float64), dev(s.u_init, torch.float64)]
    with pytest.raises(px.PxstError) as e:
        px.update_pixel_map(d, o, *args, None, small)
    assert e.value.code == -5
    ws = px.workspace(d, o)
    with pytest.raises(px.PxstError) as e:
        px.update_pixel_map(d, px.Options(-1, 2, True), *args, None, ws)
    assert e.value.code == -1
    assert px.workspace_size(px.Dims(0, 16, 16, 50, 50)) == 0
    assert px.workspace_size(px.Dims(4, 16, 16, 0, 50)) == 0
    with pytest.raises(TypeError):
        px.update_pixel_map(d, o, args[0].double(), *args[1:], None, ws)
