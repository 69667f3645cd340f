"""Parity at the full sizes of the 1-D lens scan (121 x 512 x 1536, window +-1 x +-24) and
the 2-D precision scan (400 x 1024 x 1024, window +-16 x +-16), in the launch configuration
bench.py times: the whole detector runs on the GPU, the oracle checks a sample of pixels
(one by one) and the whole reference image."""
import numpy as np
import pytest

import gen
import oracle
import parity
from gpu_util import gpu_make_object_map, gpu_update

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _sample(M, k, seed):
    rng = np.random.default_rng(seed)
    good = np.flatnonzero(M.ravel())
    ny, nx = M.shape
    # the first and last rows and columns of the mask (window and coverage edges) + random
    yy, xx = np.divmod(good, nx)
    edge = good[(yy == yy.min()) | (yy == yy.max()) | (xx == xx.min()) | (xx == xx.max())]
    pick = rng.choice(good, size=min(k, good.size), replace=False)
    return np.unique(np.concatenate([pick, edge[:: max(1, edge.size // 400)]]))


_CACHE = {}


def nonsep_stripe():
    """24 rows of the 2-D precision scan's geometry at its full width, 400 frames on the
    20 x 20 grid of 4 px steps, window +-16 x +-16, with a map that couples the axes (a
    0.01 rad rotation and a shear of 1 px amplitude on top of the magnification 1.02 and the
    +-8 px cubic) and 1 % isolated bad pixels."""
    return gen.nonsep2d(n_side=20, step=4, ny=24, nx=1024, ref=(180, 1200), sigma=1.5, mag=1.02, offset=104.0,
                        theta=0.01, curl=1.0, aberr=8.0, window=16, w_sigma=400.0, seed=gen.BASE_SEED + 32,
                        name="precision2d-nonsep-24x1024")


def _scan(name):
    if name not in _CACHE:
        _CACHE.clear()
        _CACHE[name] = nonsep_stripe() if name == "precision2d-nonsep" else gen.CONFIGS[name]()
    return _CACHE[name]


@pytest.mark.parametrize("name,k,form", [("lens1d", 3000, 0), ("precision2d", 600, 0), ("precision2d", 600, 1),
                                         ("precision2d", 600, 2), ("precision2d-nonsep", 2000, 0),
                                         ("precision2d-nonsep", 2000, 1), ("precision2d-nonsep", 2000, 2)],
                         ids=["lens1d-fp32", "precision2d-fp32", "precision2d-bf16", "precision2d-tf32",
                              "precision2d-nonsep-fp32", "precision2d-nonsep-bf16", "precision2d-nonsep-tf32"])
def test_full_size(name, k, form):
    s = _scan(name)
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    if form == 0:
        Ig, wg = gpu_make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
        print(name, "make_object_map", parity.check_omap(Ig, wg, Io, wo))
    I32, w32 = Io.astype(np.float32), wo.astype(np.float32)
    inp = dict(frames=s.frames, W=s.W, M=s.M, Iref=I32.astype(np.float64), w=w32.astype(np.float64),
               delta=s.delta, u=s.u_init, window=s.window)
    ug_i, eg_i, n_exact = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window,
                                     quadratic=False, return_exact=True, form=form)
    ug_q, eg_q = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=True,
                            form=form)
    pix = _sample(s.M, k, gen.BASE_SEED + 55)
    rep = parity.check_update(inp, pix, ug_i.reshape(2, -1)[:, pix], eg_i.ravel()[pix],
                              ug_q.reshape(2, -1)[:, pix], eg_q.ravel()[pix])
    print(name, "form", form, "update_pixel_map", rep, "exact-rule pixels:", n_exact)
