"""The tcgen05 contraction (TMA 128-byte-swizzled operands, MMA into TMEM, tcgen05.ld
read-back) against a float64 product of the same rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,K", [(1, 64), (1, 448), (2, 32), (2, 416)])
def test_tensor_contraction(form, K):
    import torch
    import paper_2003_12726_gb300 as px
    g = torch.Generator().manual_seed(1234 + K + form)
    A = torch.randn(128, K, generator=g) * 0.3
    B = torch.randn(256, K, generator=g) * 0.3
    dt = torch.bfloat16 if form == px.FORM_BF16 else torch.float32
    Ad, Bd = A.to(dt).cuda(), B.to(dt).cuda()
    D, status = px.tensor_check(form, Ad, Bd)
    assert status == 0
    Ar = Ad.float().cpu().double().numpy()
    Br = Bd.float().cpu().double().numpy()
    ref = Ar @ Br.T
    D = D.cpu().numpy()
    if form == px.FORM_TF32:
        # TF32 keeps 10 mantissa bits of each input: every product is within 2^-9 of its
        # exact value relative to |a||b|, plus FP32 accumulation
        bound = 2.0 ** -9 * (np.abs(Ar) @ np.abs(Br).T) + 1e-5
        assert np.all(np.abs(D - ref) <= bound), np.max(np.abs(D - ref) / bound)
    else:
        # BF16 inputs are exact in FP32: only the FP32 accumulation differs
        assert np.max(np.abs(D - ref)) < 1e-5 * np.sqrt(K) + 1e-5


def _ragged2d():
    from test_gpu_parity import ragged2d
    return ragged2d()


SCANS = {
    "small": lambda: __import__("gen").config_small(),
    "ragged2d": _ragged2d,
    "lens1d-48x768": lambda: __import__("gen").config_lens1d(ny=48, nx=768),
    "2d-100x96": lambda: __import__("gen").tiny2d(n_side=10, det=96, step=4, ref=200, sigma=1.5, mag=1.02,
                                                  offset=50.0, aberr=3.0, window=8,
                                                  seed=__import__("gen").BASE_SEED + 61),
    # axes coupled by a rotation and a shear (a tile's union of windows grows past its rows
    # and columns) with 1 % isolated bad pixels; fractional translations on both axes
    "nonsep2d": lambda: __import__("gen").nonsep2d(),
    "nonsep2d-100x96": lambda: __import__("gen").nonsep2d(n_side=10, det=96, step=4, ref=230, sigma=1.5, mag=1.02,
                                                          offset=60.0, theta=0.08, curl=1.5, aberr=3.0, window=8,
                                                          jitter=0.7, seed=__import__("gen").BASE_SEED + 63),
    # more frames than the rescore stages per slice (512)
    "2d-625x40": lambda: __import__("gen").tiny2d(n_side=25, det=40, step=2, ref=160, sigma=1.5, mag=1.02,
                                                  offset=60.0, aberr=2.0, window=5,
                                                  seed=__import__("gen").BASE_SEED + 62),
}


@pytest.fixture(scope="module", params=sorted(SCANS))
def tscan(request):
    return SCANS[request.param]()


def _inputs(s, hole):
    import oracle
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    I32, w32 = Io.astype(np.float32), wo.astype(np.float32)
    if hole:
        # an uncovered patch inside the reference: candidates reading it lose frames, and
        # their pixels are ranked again with the variance over their valid frames
        Ry, Rx = s.ref_shape
        w32[Ry // 2 - 3:Ry // 2 + 3, Rx // 2 - 4:Rx // 2 + 4] = 0.0
        I32[w32 == 0] = 0.0
    inp = dict(frames=s.frames, W=s.W, M=s.M, Iref=I32.astype(np.float64), w=w32.astype(np.float64),
               delta=s.delta, u=s.u_init, window=s.window)
    return inp, I32, w32


@pytest.mark.parametrize("hole", [False, True], ids=["covered", "hole"])
@pytest.mark.parametrize("form", [1, 2], ids=["bf16", "tf32"])
def test_tensor_form_parity(tscan, form, hole):
    """BF16 / TF32 ranking on the tensor cores (the masked ranking for pixels with candidates
    not valid in every frame) + exact FP32 evaluation of the best few against the FP64 oracle,
    with the same tolerances as the FP32 form."""
    import parity
    from gpu_util import gpu_update
    s = tscan
    inp, I32, w32 = _inputs(s, hole)
    ug_i, eg_i, n_slow = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=False,
                                    return_exact=True, form=form)
    ug_q, eg_q = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=True, form=form)
    pix = np.flatnonzero(s.M.ravel())
    rep = parity.check_update(inp, pix, ug_i.reshape(2, -1)[:, pix], eg_i.ravel()[pix],
                              ug_q.reshape(2, -1)[:, pix], eg_q.ravel()[pix])
    off = s.M == 0
    assert np.array_equal(ug_q[:, off], s.u_init[:, off])
    assert np.all(np.isnan(eg_q[off]))
    if hole:
        assert n_slow > 0
    print(s.name, "form", form, "hole" if hole else "", rep, "masked-rule pixels:", n_slow)


@pytest.mark.parametrize("form", [1, 2], ids=["bf16", "tf32"])
def test_tensor_form_deterministic(tscan, form):
    """Repeated calls of a tensor form give bit-identical maps and errors."""
    from gpu_util import gpu_update
    s = tscan
    _, I32, w32 = _inputs(s, True)
    runs = [gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=True, form=form)
            for _ in range(3)]
    for k in (1, 2):
        assert np.array_equal(runs[0][0], runs[k][0])
        assert np.array_equal(runs[0][1], runs[k][1], equal_nan=True)


@pytest.mark.parametrize("tile", [1, 2], ids=["4x32-4x64", "2x64-2x128"])
def test_tensor_tile_shapes(tscan, tile):
    """The other pixel-tile / candidate-chunk shapes of the tensor search (BF16) against the
    oracle, on the scans with uncovered reference pixels."""
    import parity
    from gpu_util import gpu_update
    s = tscan
    inp, I32, w32 = _inputs(s, True)
    ug_i, eg_i = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=False, form=1,
                            tile=tile)
    ug_q, eg_q = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=True, form=1,
                            tile=tile)
    pix = np.flatnonzero(s.M.ravel())
    rep = parity.check_update(inp, pix, ug_i.reshape(2, -1)[:, pix], eg_i.ravel()[pix],
                              ug_q.reshape(2, -1)[:, pix], eg_q.ravel()[pix])
    print(s.name, "tile", tile, rep)


@pytest.mark.parametrize("form", [1, 2], ids=["bf16", "tf32"])
def test_tensor_iterate_parity(tscan, form):
    """A whole iteration in a tensor form (pxst_iterate) with the full criterion: the
    reference image against the oracle's, the map update against the oracle's update on the
    GPU's own reference image."""
    import parity
    from gpu_util import gpu_iteration_pair
    s = tscan
    g_int, g_q = gpu_iteration_pair(s, s.u_init, form=form)
    print(s.name, "form", form, parity.check_iteration(s, s.u_init, g_int, g_q))
