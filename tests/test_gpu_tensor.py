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


SCANS = {
    "small": lambda: __import__("gen").config_small(),
    "lens1d-48x768": lambda: __import__("gen").config_lens1d(ny=48, nx=768),
    "2d-100x96": lambda: __import__("gen").tiny2d(n_side=10, det=96, step=4, ref=200, sigma=1.5, mag=1.02,
                                                  offset=50.0, aberr=3.0, window=8,
                                                  seed=__import__("gen").BASE_SEED + 61),
}


@pytest.fixture(scope="module", params=sorted(SCANS))
def tscan(request):
    return SCANS[request.param]()


@pytest.mark.parametrize("form", [1, 2], ids=["bf16", "tf32"])
def test_tensor_form_parity(tscan, form):
    """BF16 / TF32 ranking on the tensor cores + exact FP32 evaluation of the best 4 (and of
    every candidate of pixels touching invalid reference pixels) against the FP64 oracle,
    with the same tolerances as the FP32 form."""
    import oracle
    import parity
    from gpu_util import gpu_update
    s = tscan
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    I32, w32 = Io.astype(np.float32), wo.astype(np.float32)
    inp = dict(frames=s.frames, W=s.W, M=s.M, Iref=I32.astype(np.float64), w=w32.astype(np.float64),
               delta=s.delta, u=s.u_init, window=s.window)
    ug_i, eg_i = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=False, form=form)
    ug_q, eg_q = gpu_update(s.frames, s.W, s.M, I32, w32, s.delta, s.u_init, s.window, quadratic=True, form=form)
    pix = np.flatnonzero(s.M.ravel())
    rep = parity.check_update(inp, pix, ug_i.reshape(2, -1)[:, pix], eg_i.ravel()[pix],
                              ug_q.reshape(2, -1)[:, pix], eg_q.ravel()[pix])
    print(s.name, "form", form, rep)
