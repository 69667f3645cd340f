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
    if form == px.FORM_TF32:
        # TF32 keeps 10 mantissa bits: compare against the product of the truncated inputs,
        # with a tolerance covering either rounding of the inputs
        ref = Ar @ Br.T
        tol = 2e-3 * np.sqrt(K) * 0.09 + 1e-4
    else:
        ref = Ar @ Br.T
        tol = 1e-5 * np.sqrt(K) + 1e-5
    err = np.abs(D.cpu().numpy() - ref).max()
    assert err < tol, (err, tol)
